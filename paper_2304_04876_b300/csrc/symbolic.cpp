// Symbolic phase (Sec. V-A1 (a)): everything that depends only on the sparsity
// pattern and the partition, computed once on the host.
//
//  * nonoverlapping blocks, the interface Gamma and its vertex / edge / face
//    components (Sec. III, Fig. 1), read from the separator node planes;
//  * overlapping subdomains Omega_s' by algebraic overlap (Sec. VII: one
//    layer) at node level;
//  * the pattern of every local matrix A_s = R_s A R_s^T with the map back to
//    the entries of A (so values can be refreshed on the device);
//  * level sets of the lower and upper triangles (Sec. V-B2, V-B3) and the
//    level-sliced ELL layout the device triangular solves stream;
//  * the scatter lists that sum the overlapping local solutions in ascending
//    subdomain order;
//  * once the component ranks are known, the layout of the GDSW basis (Eq. 2)
//    as dense per-block column panels.
#include <algorithm>
#include <climits>
#include <queue>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace gdsw {

namespace {

bool fits_i32(int64_t v) { return v >= 0 && v < (int64_t(1) << 31); }

// Levels of a triangle of one subdomain's local CSR, by node: the dpn rows of
// a node (consecutive local rows) form one group that a single thread (or
// thread group) updates in order, so only couplings between different nodes
// create levels.  lower: entries j < i, rows of a node in increasing order;
// upper: entries j > i, rows of a node in decreasing order.
void build_ell(const Plan& P, int s, bool lower, int local_solver, EllPlan* E) {
  const int base = P.om_ptr[s];
  const int m = P.om_ptr[s + 1] - base;
  const int G = P.dpn;
  const int ng = m / G;
  std::vector<int> glev(ng, 0);
  int nlev = 0;
  auto off_entries = [&](int i, int& first, int& last) {
    const int r0 = P.lm_rowptr[base + i], r1 = P.lm_rowptr[base + i + 1];
    const int d = P.lm_diag[base + i];
    if (lower) { first = r0; last = d; } else { first = d + 1; last = r1; }
  };
  auto group_level = [&](int g) {
    int l = 0;
    for (int d = 0; d < G; ++d) {
      int a, b;
      off_entries(g * G + d, a, b);
      for (int e = a; e < b; ++e) {
        const int gj = P.lm_col[e] / G;
        if (gj != g) l = std::max(l, glev[gj] + 1);
      }
    }
    glev[g] = l;
    nlev = std::max(nlev, l + 1);
  };
  if (lower) for (int g = 0; g < ng; ++g) group_level(g);
  else for (int g = ng - 1; g >= 0; --g) group_level(g);
  std::vector<int> lev(m);
  for (int i = 0; i < m; ++i) lev[i] = glev[i / G];
  if (m == 0) nlev = 0;
  // bucket rows by level, ascending row inside a level
  std::vector<int> cnt(nlev + 1, 0);
  for (int i = 0; i < m; ++i) cnt[lev[i] + 1]++;
  for (int l = 0; l < nlev; ++l) cnt[l + 1] += cnt[l];
  std::vector<int> order(m);
  {
    // rows of one node stay together, in the order they are solved
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int g = 0; g < ng; ++g)
      for (int d = 0; d < G; ++d) order[pos[glev[g]]++] = g * G + (lower ? d : G - 1 - d);
  }
  E->max_levels = std::max(E->max_levels, nlev);
  for (int l = 0; l < nlev; ++l) {
    const int nr = cnt[l + 1] - cnt[l];
    int K = 0;
    for (int t = 0; t < nr; ++t) {
      int a, b;
      off_entries(order[cnt[l] + t], a, b);
      K = std::max(K, b - a);
    }
    const int start = base + cnt[l];
    const int64_t off = E->slots;
    E->lev_start.push_back(start);
    E->lev_nr.push_back(nr);
    E->lev_K.push_back(K);
    E->lev_off.push_back(static_cast<int>(off));
    E->col.resize(off + int64_t(K) * nr);
    E->src.resize(off + int64_t(K) * nr);
    for (int t = 0; t < nr; ++t) {
      const int i = order[cnt[l] + t];
      E->lrows[start + t] = static_cast<uint16_t>(i);
      const int d = P.lm_diag[base + i];
      E->dsrc[start + t] = (lower && local_solver == GDSW_LOCAL_ILU0) ? -1 : d;
      int a, b;
      off_entries(i, a, b);
      E->nnz += (b - a) + 1;
      for (int k = 0; k < K; ++k) {
        const int64_t slot = off + int64_t(k) * nr + t;
        if (a + k < b) {
          const int e = a + k;
          E->col[slot] = static_cast<uint16_t>(P.lm_col[e]);
          // IC: the upper factor is L^T, read from the transposed lower entry
          E->src[slot] = (!lower && local_solver == GDSW_LOCAL_IC0) ? P.lm_tpos[e] : e;
        } else {
          E->col[slot] = static_cast<uint16_t>(i);
          E->src[slot] = -1;
        }
      }
    }
    E->slots = off + int64_t(K) * nr;
  }
}

}  // namespace

// Level-of-fill pattern of every local matrix (ILU(k), Sec. V-B): entries of
// A_s have level 0; eliminating row i with pivot p (increasing column order,
// fill included) gives (i, j), j > p, the level lev(i,p) + lev(p,j) + 1, with
// lev(p, j) the final level of row p; entries of level <= k are kept.  Fill
// entries get lm_gent = -1 (value zero before the factorisation sweeps).
gdsw_status add_level_fill(Plan* P, int k) {
  const int nsub = P->nsub;
  std::vector<int> nrowptr(P->sum_m + 1, 0), ncol, ngent, ndiag(P->sum_m, -1), nsub_ent(nsub + 1, 0);
  std::vector<uint16_t> nrow;
  ncol.reserve(P->lm_col.size() * 2);
  ngent.reserve(P->lm_col.size() * 2);
  nrow.reserve(P->lm_col.size() * 2);
  constexpr int kNone = INT32_MAX;
  std::vector<int> lev(P->max_m, kNone), orig(P->max_m, -1);
  int64_t ent = 0;
  for (int s = 0; s < nsub; ++s) {
    const int base = P->om_ptr[s], m = P->om_ptr[s + 1] - base;
    std::vector<std::vector<std::pair<int, int>>> upper(m);   // finished rows: (column > row, level)
    std::vector<int> cols;
    for (int i = 0; i < m; ++i) {
      cols.clear();
      std::priority_queue<int, std::vector<int>, std::greater<int>> heap;
      for (int e = P->lm_rowptr[base + i]; e < P->lm_rowptr[base + i + 1]; ++e) {
        const int j = P->lm_col[e];
        lev[j] = 0;
        orig[j] = P->lm_gent[e];
        cols.push_back(j);
        if (j < i) heap.push(j);
      }
      while (!heap.empty()) {
        const int piv = heap.top();
        heap.pop();
        const int lp = lev[piv];
        for (const auto& jl : upper[piv]) {
          const int nl = lp + jl.second + 1;
          if (nl > k) continue;
          const int j = jl.first;
          if (lev[j] == kNone) {
            lev[j] = nl;
            cols.push_back(j);
            if (j < i) heap.push(j);
          } else if (nl < lev[j]) {
            lev[j] = nl;
          }
        }
      }
      std::sort(cols.begin(), cols.end());
      for (int j : cols) {
        if (j == i) ndiag[base + i] = static_cast<int>(ent);
        if (j > i) upper[i].push_back({j, lev[j]});
        ncol.push_back(j);
        nrow.push_back(static_cast<uint16_t>(i));
        ngent.push_back(orig[j]);
        ++ent;
        lev[j] = kNone;
        orig[j] = -1;
      }
      if (!fits_i32(ent)) { set_error("local factors with fill too large"); return GDSW_ERR_UNSUPPORTED; }
      nrowptr[base + i + 1] = static_cast<int>(ent);
    }
    nsub_ent[s + 1] = static_cast<int>(ent);
  }
  P->lm_rowptr.swap(nrowptr);
  P->lm_col.swap(ncol);
  P->lm_row.swap(nrow);
  P->lm_gent.swap(ngent);
  P->lm_diag.swap(ndiag);
  P->lm_sub_ent.swap(nsub_ent);
  return GDSW_OK;
}

gdsw_status build_plan(const gdsw_csr* A, const gdsw_partition* part, const gdsw_options* opt,
                       bool need_levels, Plan* P) {
  if (!A || !part || !opt || !P) { set_error("null argument"); return GDSW_ERR_INVALID_ARG; }
  if (!A->rowptr || !A->colind || !A->val) { set_error("null CSR array"); return GDSW_ERR_INVALID_ARG; }
  const int n = A->n;
  const int dpn = part->dofs_per_node;
  const int dims[3] = {part->nx, part->ny, part->nz};
  if (n <= 0 || dpn <= 0 || dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) {
    set_error("non-positive size"); return GDSW_ERR_INVALID_ARG;
  }
  const int64_t nnodes64 = int64_t(dims[0]) * dims[1] * dims[2];
  if (nnodes64 * dpn != n) {
    set_error("partition has %lld unknowns, matrix %d", (long long)(nnodes64 * dpn), n);
    return GDSW_ERR_INVALID_ARG;
  }
  const int* rp = A->rowptr;
  const int* ci = A->colind;
  if (rp[0] != 0) { set_error("rowptr[0] != 0"); return GDSW_ERR_INVALID_ARG; }
  for (int i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) { set_error("rowptr not monotone at %d", i); return GDSW_ERR_INVALID_ARG; }
    bool diag = false;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      if (ci[e] < 0 || ci[e] >= n) { set_error("column out of range in row %d", i); return GDSW_ERR_INVALID_ARG; }
      if (e > rp[i] && ci[e] <= ci[e - 1]) { set_error("columns not strictly increasing in row %d", i); return GDSW_ERR_INVALID_ARG; }
      diag |= ci[e] == i;
    }
    if (!diag) { set_error("row %d has no stored diagonal", i); return GDSW_ERR_INVALID_ARG; }
  }
  P->n = n;
  P->dpn = dpn;
  P->nnz = rp[n];
  P->nnodes = static_cast<int>(nnodes64);
  const int nn = P->nnodes;

  // ---- blocks and interface (Sec. III) ----
  std::vector<int> blk[3];
  std::vector<char> onp[3];
  for (int a = 0; a < 3; ++a) {
    const int nc = part->ncut[a];
    if (nc < 0 || (nc > 0 && !part->cut[a])) { set_error("bad cut list on axis %d", a); return GDSW_ERR_INVALID_ARG; }
    for (int t = 0; t < nc; ++t) {
      const int c = part->cut[a][t];
      if (c < 0 || c >= dims[a] - 1 || (t > 0 && c <= part->cut[a][t - 1])) {
        set_error("cut %d on axis %d must be ascending in [0, %d)", c, a, dims[a] - 1);
        return GDSW_ERR_INVALID_ARG;
      }
    }
    blk[a].assign(dims[a], 0);
    onp[a].assign(dims[a], 0);
    int t = 0;
    for (int i = 0; i < dims[a]; ++i) {
      while (t < nc && part->cut[a][t] < i) ++t;
      blk[a][i] = t;
      onp[a][i] = (t < nc && part->cut[a][t] == i) ? 1 : 0;
    }
    P->nb[a] = nc + 1;
  }
  const int64_t nsub64 = int64_t(P->nb[0]) * P->nb[1] * P->nb[2];
  if (!fits_i32(nsub64)) { set_error("too many subdomains"); return GDSW_ERR_INVALID_ARG; }
  P->nsub = static_cast<int>(nsub64);
  const int nsub = P->nsub;
  P->node_sub.resize(nn);
  P->node_comp.assign(nn, -1);
  const int64_t nkeys = int64_t(8) * P->nb[0] * P->nb[1] * P->nb[2];
  std::vector<int> key2comp(nkeys, -1);
  std::vector<int> comp_key;   // per component and axis: 2*index + on_plane
  for (int k = 0; k < dims[2]; ++k)
    for (int j = 0; j < dims[1]; ++j)
      for (int i = 0; i < dims[0]; ++i) {
        const int u = i + dims[0] * (j + dims[1] * k);
        P->node_sub[u] = blk[0][i] + P->nb[0] * (blk[1][j] + P->nb[1] * blk[2][k]);
        const int np = onp[0][i] + onp[1][j] + onp[2][k];
        if (np == 0) continue;
        const int64_t key = (2 * blk[0][i] + onp[0][i]) +
                            int64_t(2 * P->nb[0]) * ((2 * blk[1][j] + onp[1][j]) +
                                                     int64_t(2 * P->nb[1]) * (2 * blk[2][k] + onp[2][k]));
        int c = key2comp[key];
        if (c < 0) {
          c = key2comp[key] = P->ncomp++;
          P->comp_type.push_back(np);
          comp_key.push_back(2 * blk[0][i] + onp[0][i]);
          comp_key.push_back(2 * blk[1][j] + onp[1][j]);
          comp_key.push_back(2 * blk[2][k] + onp[2][k]);
        }
        P->node_comp[u] = c;
      }
  const int ncomp = P->ncomp;
  // component and interior dof lists (natural order, node-major)
  P->comp_ptr.assign(ncomp + 1, 0);
  P->int_ptr.assign(nsub + 1, 0);
  for (int u = 0; u < nn; ++u) {
    if (P->node_comp[u] >= 0) P->comp_ptr[P->node_comp[u] + 1] += dpn;
    else P->int_ptr[P->node_sub[u] + 1] += dpn;
  }
  for (int c = 0; c < ncomp; ++c) P->comp_ptr[c + 1] += P->comp_ptr[c];
  for (int s = 0; s < nsub; ++s) P->int_ptr[s + 1] += P->int_ptr[s];
  P->comp_dofs.resize(P->comp_ptr[ncomp]);
  P->int_dofs.resize(P->int_ptr[nsub]);
  P->dof_comp.assign(n, -1);
  P->dof_comprow.assign(n, -1);
  P->dof_introw.assign(n, -1);
  {
    std::vector<int> cpos(P->comp_ptr.begin(), P->comp_ptr.end() - 1);
    std::vector<int> ipos(P->int_ptr.begin(), P->int_ptr.end() - 1);
    for (int u = 0; u < nn; ++u) {
      const int c = P->node_comp[u];
      for (int d = 0; d < dpn; ++d) {
        const int g = dpn * u + d;
        if (c >= 0) {
          P->dof_comp[g] = c;
          P->dof_comprow[g] = cpos[c] - P->comp_ptr[c];
          P->comp_dofs[cpos[c]++] = g;
        } else {
          const int s = P->node_sub[u];
          P->dof_introw[g] = ipos[s] - P->int_ptr[s];
          P->int_dofs[ipos[s]++] = g;
        }
      }
    }
  }

  // ---- coarse-space owners ----
  // A vertex lies in the closure of component c when, on every axis, it is on
  // c's plane if c lies on a plane there, and on one of the two planes bounding
  // c's block otherwise (block b lies between planes b-1 and b).
  P->own_ptr.assign(ncomp + 1, 0);
  P->own_comp.clear();
  P->own_w.clear();
  {
    std::vector<int> vert_of(int64_t(part->ncut[0]) * part->ncut[1] * part->ncut[2] + 1, -1);
    for (int c = 0; c < ncomp; ++c)
      if (P->comp_type[c] == 3)
        vert_of[(comp_key[3 * c] / 2) + int64_t(part->ncut[0]) * ((comp_key[3 * c + 1] / 2) +
                                                                 int64_t(part->ncut[1]) * (comp_key[3 * c + 2] / 2))] = c;
    const bool reduced = opt->coarse == GDSW_COARSE_RGDSW;
    for (int c = 0; c < ncomp; ++c) {
      if (!reduced || P->comp_type[c] == 3) {
        P->own_comp.push_back(c);
        P->own_w.push_back(1.0);
      } else {
        std::vector<int> ch[3];
        for (int a = 0; a < 3; ++a) {
          const int key = comp_key[3 * c + a], idx = key / 2;
          if (key & 1) ch[a].push_back(idx);
          else for (int q : {idx - 1, idx}) if (q >= 0 && q < part->ncut[a]) ch[a].push_back(q);
        }
        std::vector<int> vs;
        for (int x : ch[0]) for (int y : ch[1]) for (int z : ch[2]) {
          const int v = vert_of[x + int64_t(part->ncut[0]) * (y + int64_t(part->ncut[1]) * z)];
          if (v >= 0) vs.push_back(v);
        }
        if (vs.empty()) {
          set_error("reduced GDSW needs a vertex in the closure of every interface component");
          return GDSW_ERR_UNSUPPORTED;
        }
        std::sort(vs.begin(), vs.end());
        for (int v : vs) {
          P->own_comp.push_back(v);
          P->own_w.push_back(1.0 / vs.size());
        }
      }
      P->own_ptr[c + 1] = static_cast<int>(P->own_comp.size());
    }
  }

  // ---- node graph and overlapping subdomains ----
  std::vector<int> nptr(nn + 1, 0), nadj;
  {
    std::vector<int> mark(nn, -1);
    nadj.reserve(static_cast<size_t>(P->nnz / (int64_t(dpn) * dpn) + nn));
    for (int u = 0; u < nn; ++u) {
      for (int d = 0; d < dpn; ++d) {
        const int g = dpn * u + d;
        for (int e = rp[g]; e < rp[g + 1]; ++e) {
          const int v = ci[e] / dpn;
          if (mark[v] != u) { mark[v] = u; nadj.push_back(v); }
        }
      }
      nptr[u + 1] = static_cast<int>(nadj.size());
    }
  }
  std::vector<int> sub_nptr(nsub + 1, 0), sub_nodes(nn);
  for (int u = 0; u < nn; ++u) sub_nptr[P->node_sub[u] + 1]++;
  for (int s = 0; s < nsub; ++s) sub_nptr[s + 1] += sub_nptr[s];
  {
    std::vector<int> pos(sub_nptr.begin(), sub_nptr.end() - 1);
    for (int u = 0; u < nn; ++u) sub_nodes[pos[P->node_sub[u]]++] = u;
  }
  const int delta = std::max(0, opt->overlap);
  P->om_ptr.assign(nsub + 1, 0);
  std::vector<std::vector<int>> om_nodes(nsub);
  {
    std::vector<int> mark(nn, -1);
    for (int s = 0; s < nsub; ++s) {
      std::vector<int>& list = om_nodes[s];
      for (int q = sub_nptr[s]; q < sub_nptr[s + 1]; ++q) { list.push_back(sub_nodes[q]); mark[sub_nodes[q]] = s; }
      size_t front0 = 0;
      for (int layer = 0; layer < delta; ++layer) {
        const size_t front1 = list.size();
        for (size_t q = front0; q < front1; ++q) {
          const int u = list[q];
          for (int e = nptr[u]; e < nptr[u + 1]; ++e) {
            const int v = nadj[e];
            if (mark[v] != s) { mark[v] = s; list.push_back(v); }
          }
        }
        front0 = front1;
      }
      std::sort(list.begin(), list.end());
      if (!fits_i32(int64_t(P->om_ptr[s]) + int64_t(list.size()) * dpn)) {
        set_error("overlap too large"); return GDSW_ERR_UNSUPPORTED;
      }
      P->om_ptr[s + 1] = P->om_ptr[s] + static_cast<int>(list.size()) * dpn;
    }
  }
  P->sum_m = P->om_ptr[nsub];
  P->om_dofs.resize(P->sum_m);
  P->max_m = 0;
  for (int s = 0; s < nsub; ++s) {
    int q = P->om_ptr[s];
    for (int u : om_nodes[s])
      for (int d = 0; d < dpn; ++d) P->om_dofs[q++] = dpn * u + d;
    P->max_m = std::max(P->max_m, P->om_ptr[s + 1] - P->om_ptr[s]);
  }
  om_nodes.clear();
  if (P->max_m > 65535) {
    set_error("subdomain with %d unknowns exceeds the 16-bit local index limit", P->max_m);
    return GDSW_ERR_UNSUPPORTED;
  }

  // ---- local matrices, bandwidths, interior adjacency ----
  P->lm_rowptr.assign(P->sum_m + 1, 0);
  P->lm_diag.assign(P->sum_m, -1);
  P->lm_sub_ent.assign(nsub + 1, 0);
  P->om_bw.assign(nsub, 0);
  P->int_bw.assign(nsub, 0);
  P->int_adj.assign(nsub, {});
  {
    std::vector<int> g2l(n, -1);
    int64_t ent = 0;
    for (int s = 0; s < nsub; ++s) {
      const int base = P->om_ptr[s], m = P->om_ptr[s + 1] - base;
      for (int i = 0; i < m; ++i) g2l[P->om_dofs[base + i]] = i;
      int bw = 0;
      for (int i = 0; i < m; ++i) {
        const int g = P->om_dofs[base + i];
        for (int e = rp[g]; e < rp[g + 1]; ++e) {
          const int j = g2l[ci[e]];
          if (j < 0) continue;
          if (j == i) P->lm_diag[base + i] = static_cast<int>(ent);
          P->lm_col.push_back(j);
          P->lm_row.push_back(static_cast<uint16_t>(i));
          P->lm_gent.push_back(e);
          bw = std::max(bw, std::abs(i - j));
          ++ent;
        }
        if (!fits_i32(ent)) { set_error("local matrices too large"); return GDSW_ERR_UNSUPPORTED; }
        P->lm_rowptr[base + i + 1] = static_cast<int>(ent);
      }
      P->lm_sub_ent[s + 1] = static_cast<int>(ent);
      P->om_bw[s] = bw;
      for (int i = 0; i < m; ++i) g2l[P->om_dofs[base + i]] = -1;
    }
    // interior bandwidth and adjacent components
    for (int s = 0; s < nsub; ++s) {
      int bw = 0;
      std::vector<int>& adj = P->int_adj[s];
      for (int q = P->int_ptr[s]; q < P->int_ptr[s + 1]; ++q) {
        const int g = P->int_dofs[q];
        const int i = P->dof_introw[g];
        for (int e = rp[g]; e < rp[g + 1]; ++e) {
          const int c = ci[e];
          if (P->dof_comp[c] >= 0) { adj.push_back(P->dof_comp[c]); continue; }
          if (P->node_sub[c / dpn] != s) {
            set_error("interiors of subdomains %d and %d are coupled: the separator planes do "
                      "not split the matrix graph", s, P->node_sub[c / dpn]);
            return GDSW_ERR_INVALID_ARG;
          }
          bw = std::max(bw, std::abs(i - P->dof_introw[c]));
        }
      }
      std::sort(adj.begin(), adj.end());
      adj.erase(std::unique(adj.begin(), adj.end()), adj.end());
      P->int_bw[s] = bw;
    }
  }
  // IC(k)/ILU(k): widen the local patterns by the level-k fill
  if (opt->fill_level > 0 && opt->local_solver != GDSW_LOCAL_EXACT) GDSW_TRY(add_level_fill(P, opt->fill_level));
  // transposed positions (structural symmetry is required)
  P->lm_tpos.assign(P->lm_col.size(), -1);
  for (int s = 0; s < nsub; ++s) {
    const int base = P->om_ptr[s], m = P->om_ptr[s + 1] - base;
    for (int i = 0; i < m; ++i) {
      for (int e = P->lm_rowptr[base + i]; e < P->lm_rowptr[base + i + 1]; ++e) {
        const int j = P->lm_col[e];
        const int* b0 = P->lm_col.data() + P->lm_rowptr[base + j];
        const int* b1 = P->lm_col.data() + P->lm_rowptr[base + j + 1];
        const int* f = std::lower_bound(b0, b1, i);
        if (f == b1 || *f != i) {
          set_error("matrix pattern is not structurally symmetric");
          return GDSW_ERR_INVALID_ARG;
        }
        P->lm_tpos[e] = static_cast<int>(f - P->lm_col.data());
      }
    }
  }

  // ---- level-sliced ELL of the triangles ----
  if (need_levels) {
    for (EllPlan* E : {&P->L, &P->U}) {
      E->sub_lev.assign(nsub + 1, 0);
      E->lrows.assign(P->sum_m, 0);
      E->dsrc.assign(P->sum_m, -1);
    }
    for (int s = 0; s < nsub; ++s) {
      build_ell(*P, s, true, opt->local_solver, &P->L);
      P->L.sub_lev[s + 1] = static_cast<int>(P->L.lev_nr.size());
      build_ell(*P, s, false, opt->local_solver, &P->U);
      P->U.sub_lev[s + 1] = static_cast<int>(P->U.lev_nr.size());
      if (!fits_i32(P->L.slots) || !fits_i32(P->U.slots)) {
        set_error("factor too large"); return GDSW_ERR_UNSUPPORTED;
      }
    }
  }

  // ---- scatter lists per dof (ascending subdomain) ----
  P->pull_dof_ptr.assign(n + 1, 0);
  for (int64_t q = 0; q < P->sum_m; ++q) P->pull_dof_ptr[P->om_dofs[q] + 1]++;
  for (int g = 0; g < n; ++g) P->pull_dof_ptr[g + 1] += P->pull_dof_ptr[g];
  P->pull_dof_pos.resize(P->sum_m);
  {
    std::vector<int> pos(P->pull_dof_ptr.begin(), P->pull_dof_ptr.end() - 1);
    for (int64_t q = 0; q < P->sum_m; ++q) P->pull_dof_pos[pos[P->om_dofs[q]]++] = static_cast<int>(q);
  }
  P->nprob = 1;
  P->prob_dof_ptr = {0, n};
  P->comp_prob.assign(P->ncomp, 0);
  return GDSW_OK;
}

gdsw_status merge_plans(std::vector<Plan>& parts, Plan* M) {
  if (parts.empty()) { set_error("empty batch"); return GDSW_ERR_INVALID_ARG; }
  Plan& o = *M;
  o = Plan();
  o.dpn = parts[0].dpn;
  o.nprob = static_cast<int>(parts.size());
  o.prob_dof_ptr.assign(o.nprob + 1, 0);
  int64_t n = 0, nnodes = 0, nnz = 0, sum_m = 0, nent = 0, nsub = 0, ncomp = 0;
  int64_t levL = 0, levU = 0, slotsL = 0, slotsU = 0;
  for (const Plan& p : parts) {
    if (p.dpn != o.dpn) { set_error("batch members must have the same unknowns per node"); return GDSW_ERR_INVALID_ARG; }
    n += p.n; nnodes += p.nnodes; nnz += p.nnz; sum_m += p.sum_m; nent += p.lm_col.size();
    nsub += p.nsub; ncomp += p.ncomp;
    levL += p.L.lev_nr.size(); levU += p.U.lev_nr.size(); slotsL += p.L.slots; slotsU += p.U.slots;
  }
  if (n >= (int64_t(1) << 31) || nnz >= (int64_t(1) << 31) || nent >= (int64_t(1) << 31) ||
      sum_m >= (int64_t(1) << 31) || slotsL >= (int64_t(1) << 31) || slotsU >= (int64_t(1) << 31)) {
    set_error("batch too large for 32-bit indices"); return GDSW_ERR_UNSUPPORTED;
  }
  o.n = static_cast<int>(n); o.nnodes = static_cast<int>(nnodes); o.nnz = nnz;
  o.nsub = static_cast<int>(nsub); o.ncomp = static_cast<int>(ncomp); o.sum_m = sum_m;
  o.om_ptr.assign(1, 0); o.int_ptr.assign(1, 0); o.comp_ptr.assign(1, 0);
  o.lm_rowptr.assign(1, 0); o.lm_sub_ent.assign(1, 0); o.pull_dof_ptr.assign(1, 0);
  for (EllPlan* E : {&o.L, &o.U}) E->sub_lev.assign(1, 0);
  int doff = 0, noff = 0, soff = 0, coff = 0, moff = 0, eoff = 0, goff = 0;
  int lvL = 0, lvU = 0, slL = 0, slU = 0;
  for (int pi = 0; pi < o.nprob; ++pi) {
    Plan& p = parts[pi];
    auto add = [](std::vector<int>& dst, const std::vector<int>& src, int off, bool keep_neg) {
      for (int v : src) dst.push_back((keep_neg && v < 0) ? v : v + off);
    };
    add(o.node_sub, p.node_sub, soff, false);
    add(o.node_comp, p.node_comp, coff, true);
    o.comp_type.insert(o.comp_type.end(), p.comp_type.begin(), p.comp_type.end());
    add(o.comp_dofs, p.comp_dofs, doff, false);
    add(o.int_dofs, p.int_dofs, doff, false);
    add(o.om_dofs, p.om_dofs, doff, false);
    add(o.dof_comp, p.dof_comp, coff, true);
    o.dof_comprow.insert(o.dof_comprow.end(), p.dof_comprow.begin(), p.dof_comprow.end());
    o.dof_introw.insert(o.dof_introw.end(), p.dof_introw.begin(), p.dof_introw.end());
    for (int q = 1; q < static_cast<int>(p.lm_rowptr.size()); ++q) o.lm_rowptr.push_back(p.lm_rowptr[q] + eoff);
    o.lm_col.insert(o.lm_col.end(), p.lm_col.begin(), p.lm_col.end());
    o.lm_row.insert(o.lm_row.end(), p.lm_row.begin(), p.lm_row.end());
    add(o.lm_gent, p.lm_gent, goff, true);
    add(o.lm_tpos, p.lm_tpos, eoff, false);
    add(o.lm_diag, p.lm_diag, eoff, false);
    for (int q = 1; q < static_cast<int>(p.lm_sub_ent.size()); ++q) o.lm_sub_ent.push_back(p.lm_sub_ent[q] + eoff);
    struct Side { EllPlan* dst; EllPlan* src; int* lv; int* sl; };
    Side sides[2] = {{&o.L, &p.L, &lvL, &slL}, {&o.U, &p.U, &lvU, &slU}};
    for (Side& sd : sides) {
      EllPlan& D = *sd.dst;
      EllPlan& S = *sd.src;
      for (size_t q = 1; q < S.sub_lev.size(); ++q) D.sub_lev.push_back(S.sub_lev[q] + *sd.lv);
      add(D.lev_start, S.lev_start, moff, false);
      D.lev_nr.insert(D.lev_nr.end(), S.lev_nr.begin(), S.lev_nr.end());
      D.lev_K.insert(D.lev_K.end(), S.lev_K.begin(), S.lev_K.end());
      add(D.lev_off, S.lev_off, *sd.sl, false);
      D.lrows.insert(D.lrows.end(), S.lrows.begin(), S.lrows.end());
      D.col.insert(D.col.end(), S.col.begin(), S.col.end());
      add(D.src, S.src, eoff, true);
      add(D.dsrc, S.dsrc, eoff, true);
      D.nnz += S.nnz;
      D.slots += S.slots;
      D.max_levels = std::max(D.max_levels, S.max_levels);
      *sd.lv += static_cast<int>(S.lev_nr.size());
      *sd.sl += static_cast<int>(S.slots);
    }
    for (const std::vector<int>& adj : p.int_adj) {
      std::vector<int> a;
      for (int c : adj) a.push_back(c + coff);
      o.int_adj.push_back(a);
    }
    o.int_bw.insert(o.int_bw.end(), p.int_bw.begin(), p.int_bw.end());
    o.om_bw.insert(o.om_bw.end(), p.om_bw.begin(), p.om_bw.end());
    for (int g = 1; g <= p.n; ++g) o.pull_dof_ptr.push_back(p.pull_dof_ptr[g] + o.pull_dof_ptr[doff]);
    add(o.pull_dof_pos, p.pull_dof_pos, moff, false);
    o.comp_prob.insert(o.comp_prob.end(), p.ncomp, pi);
    if (o.own_ptr.empty()) o.own_ptr.push_back(0);
    {
      const int oo = static_cast<int>(o.own_comp.size());
      for (size_t q = 1; q < p.own_ptr.size(); ++q) o.own_ptr.push_back(p.own_ptr[q] + oo);
    }
    add(o.own_comp, p.own_comp, coff, false);
    o.own_w.insert(o.own_w.end(), p.own_w.begin(), p.own_w.end());
    o.max_m = std::max(o.max_m, p.max_m);
    // pointer arrays from sizes
    for (int q = 0; q < p.nsub; ++q) {
      o.om_ptr.push_back(o.om_ptr.back() + p.om_ptr[q + 1] - p.om_ptr[q]);
      o.int_ptr.push_back(o.int_ptr.back() + p.int_ptr[q + 1] - p.int_ptr[q]);
    }
    doff += p.n; noff += p.nnodes; soff += p.nsub; coff += p.ncomp;
    moff += static_cast<int>(p.sum_m); eoff += static_cast<int>(p.lm_col.size()); goff += static_cast<int>(p.nnz);
    o.prob_dof_ptr[pi + 1] = doff;
    p = Plan();   // release the member's memory as soon as it is merged
  }
  // component pointers from the merged component dof lists
  o.comp_ptr.assign(o.ncomp + 1, 0);
  for (int g = 0; g < o.n; ++g)
    if (o.dof_comp[g] >= 0) o.comp_ptr[o.dof_comp[g] + 1]++;
  for (int c = 0; c < o.ncomp; ++c) o.comp_ptr[c + 1] += o.comp_ptr[c];
  (void)noff;
  return GDSW_OK;
}

gdsw_status build_supports(const Plan& P, SupportPlan* S) {
  const int ncomp = P.ncomp;
  std::vector<std::vector<std::pair<int, double>>> sup(ncomp);   // owner -> (component, weight)
  for (int c = 0; c < ncomp; ++c)
    for (int q = P.own_ptr[c]; q < P.own_ptr[c + 1]; ++q) sup[P.own_comp[q]].push_back({c, P.own_w[q]});
  S->owners.clear();
  S->supp_ptr.assign(1, 0);
  S->supp_dof.clear(); S->supp_comp.clear(); S->supp_row.clear(); S->supp_w.clear();
  for (int o = 0; o < ncomp; ++o) {
    if (sup[o].empty()) continue;
    S->owners.push_back(o);
    for (const auto& cw : sup[o]) {
      const int c = cw.first;
      for (int q = P.comp_ptr[c]; q < P.comp_ptr[c + 1]; ++q) {
        S->supp_dof.push_back(P.comp_dofs[q]);
        S->supp_comp.push_back(c);
        S->supp_row.push_back(q - P.comp_ptr[c]);
        S->supp_w.push_back(cw.second);
      }
    }
    S->supp_ptr.push_back(static_cast<int>(S->supp_dof.size()));
  }
  return GDSW_OK;
}

gdsw_status build_coarse_plan(const Plan& P, const SupportPlan& S, const std::vector<int>& comp_rank,
                              bool coarse, CoarsePlan* C) {
  const int nsub = P.nsub, ncomp = P.ncomp, n = P.n;
  C->comp_c0.assign(ncomp, 0);
  C->comp_k.assign(ncomp, 0);
  int n0 = 0;
  for (int c = 0; c < ncomp; ++c) {      // owners in component order (problem-major)
    C->comp_c0[c] = n0;
    C->comp_k[c] = coarse ? comp_rank[c] : 0;
    n0 += C->comp_k[c];
  }
  C->n0 = n0;
  C->prob_c0.assign(P.nprob + 1, 0);
  for (int c = 0; c < ncomp; ++c) C->prob_c0[P.comp_prob[c] + 1] += C->comp_k[c];
  for (int q = 0; q < P.nprob; ++q) C->prob_c0[q + 1] += C->prob_c0[q];
  // columns of each component block: its owners' columns, owners ascending
  std::vector<std::vector<int>> comp_cols(ncomp);
  for (int c = 0; c < ncomp; ++c)
    for (int q = P.own_ptr[c]; q < P.own_ptr[c + 1]; ++q) {
      const int o = P.own_comp[q];
      for (int t = 0; t < C->comp_k[o]; ++t) comp_cols[c].push_back(C->comp_c0[o] + t);
    }
  // first column of owner o inside component c's block, for every support entry
  C->supp_colpos.assign(S.supp_dof.size(), 0);
  for (size_t oi = 0; oi < S.owners.size(); ++oi) {
    const int o = S.owners[oi];
    for (int e = S.supp_ptr[oi]; e < S.supp_ptr[oi + 1]; ++e) {
      const int c = S.supp_comp[e];
      int pos = 0;
      for (int q = P.own_ptr[c]; q < P.own_ptr[c + 1] && P.own_comp[q] != o; ++q) pos += C->comp_k[P.own_comp[q]];
      C->supp_colpos[e] = pos;
    }
  }
  C->nblk = nsub + ncomp;
  const int nblk = C->nblk;
  C->brow_ptr.assign(nblk + 1, 0);
  C->bcol_ptr.assign(nblk + 1, 0);
  C->phi_off.assign(nblk + 1, 0);
  C->brow_dof.clear();
  C->brow_dof.reserve(n);
  C->bcol.clear();
  for (int b = 0; b < nblk; ++b) {
    if (b < nsub) {
      C->brow_dof.insert(C->brow_dof.end(), P.int_dofs.begin() + P.int_ptr[b],
                         P.int_dofs.begin() + P.int_ptr[b + 1]);
      std::vector<int> cols;
      for (int c : P.int_adj[b]) cols.insert(cols.end(), comp_cols[c].begin(), comp_cols[c].end());
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      C->bcol.insert(C->bcol.end(), cols.begin(), cols.end());
    } else {
      const int c = b - nsub;
      C->brow_dof.insert(C->brow_dof.end(), P.comp_dofs.begin() + P.comp_ptr[c],
                         P.comp_dofs.begin() + P.comp_ptr[c + 1]);
      C->bcol.insert(C->bcol.end(), comp_cols[c].begin(), comp_cols[c].end());
    }
    C->brow_ptr[b + 1] = static_cast<int>(C->brow_dof.size());
    C->bcol_ptr[b + 1] = static_cast<int>(C->bcol.size());
    const int64_t rows = C->brow_ptr[b + 1] - C->brow_ptr[b];
    const int64_t cols = C->bcol_ptr[b + 1] - C->bcol_ptr[b];
    C->phi_off[b + 1] = C->phi_off[b] + rows * cols;
  }
  C->phi_len = C->phi_off[nblk];
  if (static_cast<int>(C->brow_dof.size()) != n) {
    set_error("internal: blocks do not cover the unknowns"); return GDSW_ERR_INVALID_ARG;
  }
  C->dof_blk.assign(n, -1);
  C->dof_blkrow.assign(n, -1);
  for (int b = 0; b < nblk; ++b)
    for (int q = C->brow_ptr[b]; q < C->brow_ptr[b + 1]; ++q) {
      C->dof_blk[C->brow_dof[q]] = b;
      C->dof_blkrow[C->brow_dof[q]] = q - C->brow_ptr[b];
    }
  // Phi^T r chunks of at most kPhiChunkRows rows; partial slots per (chunk, column)
  constexpr int kChunkRows = kPhiChunkRows;
  C->chunk_blk.clear(); C->chunk_r0.clear(); C->chunk_r1.clear(); C->chunk_slot.clear();
  int nslot = 0;
  std::vector<std::vector<int>> col_slots(n0);
  for (int b = 0; b < nblk; ++b) {
    const int rows = C->brow_ptr[b + 1] - C->brow_ptr[b];
    const int k = C->bcol_ptr[b + 1] - C->bcol_ptr[b];
    if (k == 0) continue;
    for (int r0 = 0; r0 < rows; r0 += kChunkRows) {
      C->chunk_blk.push_back(b);
      C->chunk_r0.push_back(r0);
      C->chunk_r1.push_back(std::min(rows, r0 + kChunkRows));
      C->chunk_slot.push_back(nslot);
      for (int u = 0; u < k; ++u) col_slots[C->bcol[C->bcol_ptr[b] + u]].push_back(nslot + u);
      nslot += k;
    }
  }
  C->n_slots = nslot;
  // processing order: chunks of more than kWarpRows rows first (a CTA each),
  // then the small ones (a warp each); slots keep the (block, chunk) order, so
  // the order of the sums does not change
  {
    constexpr int kWarpRows = 256;
    std::vector<int> order(C->chunk_blk.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = static_cast<int>(q);
    std::stable_partition(order.begin(), order.end(),
                          [&](int q) { return C->chunk_r1[q] - C->chunk_r0[q] > kWarpRows; });
    C->n_cta_chunks = 0;
    for (int q : order) C->n_cta_chunks += C->chunk_r1[q] - C->chunk_r0[q] > kWarpRows;
    auto permute = [&](std::vector<int>& v) {
      std::vector<int> t(v.size());
      for (size_t q = 0; q < order.size(); ++q) t[q] = v[order[q]];
      v.swap(t);
    };
    permute(C->chunk_blk); permute(C->chunk_r0); permute(C->chunk_r1); permute(C->chunk_slot);
  }
  // slots of every coarse column in ascending (block, chunk) order
  C->cs_ptr.assign(n0 + 1, 0);
  C->cs_idx.clear();
  for (int l = 0; l < n0; ++l) {
    C->cs_idx.insert(C->cs_idx.end(), col_slots[l].begin(), col_slots[l].end());
    C->cs_ptr[l + 1] = static_cast<int>(C->cs_idx.size());
  }
  C->pos_blk.assign(n, 0);
  for (int b = 0; b < nblk; ++b)
    for (int q = C->brow_ptr[b]; q < C->brow_ptr[b + 1]; ++q) C->pos_blk[q] = b;
  // scatter lists in block-row order
  C->pull_ptr.assign(n + 1, 0);
  C->pull_pos.clear();
  C->pull_pos.reserve(P.sum_m);
  for (int q = 0; q < n; ++q) {
    const int g = C->brow_dof[q];
    for (int t = P.pull_dof_ptr[g]; t < P.pull_dof_ptr[g + 1]; ++t) C->pull_pos.push_back(P.pull_dof_pos[t]);
    C->pull_ptr[q + 1] = static_cast<int>(C->pull_pos.size());
  }
  return GDSW_OK;
}

}  // namespace gdsw
