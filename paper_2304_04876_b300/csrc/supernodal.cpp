// Symbolic phase of the multifrontal exact local solver (Sec. V-B1: exact
// local solves with a sparse direct factorisation; Sec. V-B2 lists the
// partitioned-inverse triangular solve as the alternative to substitution).
//
// Every subdomain matrix A_s is ordered by nested dissection of its graph
// (recursive bisection at a level set of a breadth-first search from a
// pseudo-peripheral node), which gives a tree of supernodes: the separators,
// and the leaf regions of at most `leaf` unknowns.  Supernode S with unknowns
// S and ancestor unknowns B(S) coupled to its subtree has the front S u B(S);
// its exact Cholesky factor columns are the dense block [L_SS; L_BS].  The
// solve uses the explicit inverse of L_SS (the partitioned inverse), so both
// triangular sweeps are dense matrix-vector products, one tree level at a
// time instead of one matrix row at a time.
//
// Everything here depends on the pattern only and runs on the host, one
// thread per group of subdomains.
#include <algorithm>
#include <cstdio>
#include <thread>

#include "internal.h"

namespace gdsw {

namespace {

// Minimum share of a region's nodes on each side of a separator level.
constexpr double kSepBalance = 0.3;

struct SubTree {
  // supernodes in postorder; node lists in local node numbering
  std::vector<std::vector<int>> sn_nodes;
  std::vector<std::vector<int>> sn_children;
};

// Nested dissection of the local node graph (adjacency adj_ptr/adj).
class Dissection {
 public:
  Dissection(int nn, const std::vector<int>& ptr, const std::vector<int>& adj, int leaf)
      : nn_(nn), ptr_(ptr), adj_(adj), leaf_(leaf), stamp_(nn, 0), lev_(nn, -1) {}

  void run(SubTree* T) {
    T_ = T;
    std::vector<int> all(nn_);
    for (int i = 0; i < nn_; ++i) all[i] = i;
    if (nn_ > 0) dissect(all);
  }

 private:
  int nn_;
  const std::vector<int>& ptr_;
  const std::vector<int>& adj_;
  int leaf_;
  std::vector<int> stamp_, lev_;
  int cur_ = 0;
  SubTree* T_ = nullptr;

  // breadth-first search inside the region marked with `mark`; fills order
  // and lev_ (distance from start), returns the largest distance
  int bfs(int start, int mark, std::vector<int>& order) {
    order.clear();
    order.push_back(start);
    lev_[start] = 0;
    stamp_[start] = mark + 1;
    int maxl = 0;
    for (size_t h = 0; h < order.size(); ++h) {
      const int u = order[h];
      for (int e = ptr_[u]; e < ptr_[u + 1]; ++e) {
        const int v = adj_[e];
        if (stamp_[v] != mark) continue;
        stamp_[v] = mark + 1;
        lev_[v] = lev_[u] + 1;
        maxl = std::max(maxl, lev_[v]);
        order.push_back(v);
      }
    }
    return maxl;
  }

  int new_mark(const std::vector<int>& region) {
    cur_ += 2;
    for (int u : region) stamp_[u] = cur_;
    return cur_;
  }

  int add_node(std::vector<int> nodes, std::vector<int> children) {
    std::sort(nodes.begin(), nodes.end());
    T_->sn_nodes.push_back(std::move(nodes));
    T_->sn_children.push_back(std::move(children));
    return static_cast<int>(T_->sn_nodes.size()) - 1;
  }

  // Returns the roots of the sub-forest built for `region`.
  std::vector<int> dissect(const std::vector<int>& region) {
    if (static_cast<int>(region.size()) <= leaf_) return {add_node(region, {})};
    // connected components: each is dissected on its own
    std::vector<int> order;
    int mark = new_mark(region);
    std::vector<std::vector<int>> comps;
    for (int u : region) {
      if (stamp_[u] != mark) continue;
      bfs(u, mark, order);
      comps.push_back(order);
    }
    if (comps.size() > 1) {
      std::vector<int> roots;
      for (auto& c : comps) {
        std::vector<int> r = dissect(c);
        roots.insert(roots.end(), r.begin(), r.end());
      }
      return roots;
    }
    // pseudo-peripheral start: restart from the farthest node a few times
    int start = region[0];
    int maxl = 0;
    for (int t = 0; t < 4; ++t) {
      mark = new_mark(region);
      maxl = bfs(start, mark, order);
      if (t < 3) start = order.back();
    }
    if (maxl < 2) return {add_node(region, {})};
    std::vector<int> cnt(maxl + 1, 0);
    for (int u : region) cnt[lev_[u]]++;
    // separator: the smallest inner level with at least kSepBalance of the
    // region on either side, else the level where the running count passes half
    const int tot = static_cast<int>(region.size());
    int best = -1, half = -1, below = 0;
    for (int l = 0; l <= maxl; ++l) {
      const int above = tot - below - cnt[l];
      if (l >= 1 && l <= maxl - 1) {
        if (half < 0 && below + cnt[l] >= (tot + 1) / 2) half = l;
        if (std::min(below, above) >= kSepBalance * tot && (best < 0 || cnt[l] < cnt[best])) best = l;
      }
      below += cnt[l];
    }
    const int mid = best >= 0 ? best : (half >= 0 ? half : 1);
    std::vector<int> sep, lo, hi;
    for (int u : region) {
      if (lev_[u] == mid) sep.push_back(u);
      else if (lev_[u] < mid) lo.push_back(u);
      else hi.push_back(u);
    }
    std::vector<int> children;
    for (auto* part : {&lo, &hi}) {
      if (part->empty()) continue;
      std::vector<int> r = dissect(*part);
      children.insert(children.end(), r.begin(), r.end());
    }
    return {add_node(std::move(sep), std::move(children))};
  }
};

// Per-subdomain result before concatenation (local supernode ids, local positions).
struct SubMf {
  int m = 0;
  std::vector<int> perm;                 // ND position -> local unknown
  std::vector<int> pos0, ns, nb, parent, height, uoff, stage;
  std::vector<char> small;               // solved by one warp from a staged panel
  std::vector<std::vector<int>> bset;    // B(S) as ND positions, ascending
  std::vector<std::vector<int>> children;
  std::vector<int> lev_ptr, lev_sn;      // supernodes by height
  std::vector<std::vector<int>> pullS;   // per ND position: arena entries
  std::vector<std::vector<std::vector<int>>> pullB;   // per supernode, per B row
  std::vector<std::vector<int>> relF;    // per supernode, per B row: row in the parent's front
  std::vector<std::vector<std::pair<int, uint32_t>>> asm_list;   // (local CSR entry, row | col << 16)
  std::vector<int64_t> stack_off;
  int64_t stack_peak = 0;
  int arena = 0, stage_max = 0, max_front = 0, max_ns = 0;
  std::string err;
};

int64_t panel_entries(int64_t ns, int64_t nb) { return ns * (ns + nb) - ns * (ns - 1) / 2; }

void build_sub(const Plan& P, int q, int leaf, int small_cap, SubMf* R) {
  const int base = P.om_ptr[q];
  const int m = P.om_ptr[q + 1] - base;
  const int G = P.dpn;
  R->m = m;
  if (m == 0) { R->lev_ptr = {0}; return; }
  if (m > 65535) { R->err = "subdomain has more than 65535 unknowns"; return; }
  const int nn = m / G;
  // node graph of A_s (true entries only)
  std::vector<int> aptr(nn + 1, 0), adj;
  {
    std::vector<int> mark(nn, -1);
    for (int g = 0; g < nn; ++g) {
      mark[g] = g;
      for (int d = 0; d < G; ++d) {
        const int i = g * G + d;
        for (int e = P.lm_rowptr[base + i]; e < P.lm_rowptr[base + i + 1]; ++e) {
          if (P.lm_gent[e] < 0) continue;
          const int h = P.lm_col[e] / G;
          if (mark[h] == g) continue;
          mark[h] = g;
          adj.push_back(h);
        }
      }
      aptr[g + 1] = static_cast<int>(adj.size());
    }
  }
  SubTree T;
  Dissection(nn, aptr, adj, std::max(1, leaf / G)).run(&T);
  const int nsn = static_cast<int>(T.sn_nodes.size());
  R->children = T.sn_children;
  // ND positions of the unknowns
  R->perm.resize(m);
  std::vector<int> pos(m);
  R->pos0.resize(nsn);
  R->ns.resize(nsn);
  {
    int p = 0;
    for (int S = 0; S < nsn; ++S) {
      R->pos0[S] = p;
      for (int g : T.sn_nodes[S])
        for (int d = 0; d < G; ++d) { R->perm[p] = g * G + d; pos[g * G + d] = p; ++p; }
      R->ns[S] = p - R->pos0[S];
    }
  }
  R->parent.assign(nsn, -1);
  for (int S = 0; S < nsn; ++S)
    for (int c : R->children[S]) R->parent[c] = S;
  // B(S): ancestor unknowns coupled to the subtree of S, in ND order
  R->bset.resize(nsn);
  R->nb.resize(nsn);
  for (int S = 0; S < nsn; ++S) {
    const int last = R->pos0[S] + R->ns[S];
    std::vector<int>& B = R->bset[S];
    for (int p = R->pos0[S]; p < last; ++p) {
      const int i = R->perm[p];
      for (int e = P.lm_rowptr[base + i]; e < P.lm_rowptr[base + i + 1]; ++e) {
        if (P.lm_gent[e] < 0) continue;
        const int t = pos[P.lm_col[e]];
        if (t >= last) B.push_back(t);
      }
    }
    for (int c : R->children[S])
      for (int t : R->bset[c])
        if (t >= last) B.push_back(t);
    std::sort(B.begin(), B.end());
    B.erase(std::unique(B.begin(), B.end()), B.end());
    R->nb[S] = static_cast<int>(B.size());
    R->max_front = std::max(R->max_front, R->ns[S] + R->nb[S]);
    R->max_ns = std::max(R->max_ns, R->ns[S]);
  }
  // heights and the level lists (postorder inside a level)
  R->height.assign(nsn, 0);
  int H = 0;
  for (int S = 0; S < nsn; ++S) {
    for (int c : R->children[S]) R->height[S] = std::max(R->height[S], R->height[c] + 1);
    H = std::max(H, R->height[S] + 1);
  }
  R->lev_ptr.assign(H + 1, 0);
  for (int S = 0; S < nsn; ++S) R->lev_ptr[R->height[S] + 1]++;
  for (int l = 0; l < H; ++l) R->lev_ptr[l + 1] += R->lev_ptr[l];
  R->lev_sn.resize(nsn);
  {
    std::vector<int> fill(R->lev_ptr.begin(), R->lev_ptr.end() - 1);
    for (int S = 0; S < nsn; ++S) R->lev_sn[fill[R->height[S]]++] = S;
  }
  // a supernode is small when one warp holds its rows (and at most four B rows
  // per lane) and its panel fits the warp's staging buffer
  R->small.assign(nsn, 0);
  for (int S = 0; S < nsn; ++S)
    R->small[S] = R->ns[S] <= kMfSmall && R->nb[S] <= kMfSmallNb &&
                  (panel_entries(R->ns[S], R->nb[S]) + 7) / 8 * 8 <= small_cap;
  // stage offsets (rows of the large supernodes of a level, in order) and the
  // arena: u_S lives from its own level to its parent's; first fit over
  // address-ordered free blocks
  R->stage.assign(nsn, 0);
  R->uoff.assign(nsn, 0);
  {
    std::vector<std::pair<int, int>> used;       // (offset, size), sorted by offset
    std::vector<std::vector<int>> free_at(H + 1);
    for (int l = 0; l < H; ++l) {
      for (int S : free_at[l]) {
        auto it = std::find_if(used.begin(), used.end(), [&](const std::pair<int, int>& b) {
          return b.first == R->uoff[S] && b.second == R->nb[S]; });
        if (it != used.end()) used.erase(it);
      }
      int rows = 0;
      for (int k = R->lev_ptr[l]; k < R->lev_ptr[l + 1]; ++k) {
        const int S = R->lev_sn[k];
        if (!R->small[S]) {
          R->stage[S] = rows;
          rows += R->ns[S];
        }
        if (R->nb[S] == 0) continue;
        int at = 0;
        size_t ins = 0;
        for (; ins < used.size(); ++ins) {
          if (used[ins].first - at >= R->nb[S]) break;
          at = std::max(at, used[ins].first + used[ins].second);
        }
        R->uoff[S] = at;
        used.insert(used.begin() + ins, {at, R->nb[S]});
        R->arena = std::max(R->arena, at + R->nb[S]);
        const int par = R->parent[S];
        free_at[par >= 0 ? R->height[par] + 1 : l + 1].push_back(S);
      }
      R->stage_max = std::max(R->stage_max, rows);
    }
  }
  if (R->arena > 65535) { R->err = "update vectors of a subdomain exceed 65535 entries"; return; }
  // pull lists and the rows of each child's B in its parent's front
  R->pullS.assign(m, {});
  R->pullB.resize(nsn);
  R->relF.resize(nsn);
  for (int S = 0; S < nsn; ++S) R->pullB[S].assign(R->nb[S], {});
  for (int S = 0; S < nsn; ++S) {
    const int last = R->pos0[S] + R->ns[S];
    const std::vector<int>& BS = R->bset[S];
    for (int c : R->children[S]) {
      const std::vector<int>& Bc = R->bset[c];
      R->relF[c].resize(Bc.size());
      for (size_t r = 0; r < Bc.size(); ++r) {
        const int t = Bc[r];
        const int src = R->uoff[c] + static_cast<int>(r);
        if (t < last) {
          R->pullS[t].push_back(src);
          R->relF[c][r] = t - R->pos0[S];
        } else {
          const int k = static_cast<int>(std::lower_bound(BS.begin(), BS.end(), t) - BS.begin());
          R->pullB[S][k].push_back(src);
          R->relF[c][r] = R->ns[S] + k;
        }
      }
    }
  }
  // assembly of A_s into the fronts: entry (i, j), pos i >= pos j, j in S
  R->asm_list.resize(nsn);
  for (int S = 0; S < nsn; ++S) {
    const int p0 = R->pos0[S], last = p0 + R->ns[S];
    const std::vector<int>& BS = R->bset[S];
    for (int p = p0; p < last; ++p) {
      const int j = R->perm[p];
      for (int e = P.lm_rowptr[base + j]; e < P.lm_rowptr[base + j + 1]; ++e) {
        if (P.lm_gent[e] < 0) continue;
        const int t = pos[P.lm_col[e]];
        if (t < p) continue;
        const int fr = t < last ? t - p0
                                : R->ns[S] + static_cast<int>(std::lower_bound(BS.begin(), BS.end(), t) - BS.begin());
        R->asm_list[S].push_back({e, uint32_t(fr) | (uint32_t(p - p0) << 16)});
      }
    }
  }
  // update matrices on a stack (postorder: a node's children are on top)
  R->stack_off.assign(nsn, 0);
  int64_t sp = 0;
  for (int S = 0; S < nsn; ++S) {
    int64_t at = sp;
    for (int c : R->children[S]) at = std::min(at, R->stack_off[c]);
    R->stack_off[S] = at;
    sp = at + int64_t(R->nb[S]) * R->nb[S];
    R->stack_peak = std::max(R->stack_peak, sp);
  }
}

}  // namespace

gdsw_status build_mf_plan(const Plan& P, int leaf, int small_cap, MfPlan* M) {
  const int nsub = P.nsub;
  std::vector<SubMf> subs(nsub);
  unsigned hw = std::thread::hardware_concurrency();
  const int nth = static_cast<int>(std::max(1u, std::min<unsigned>(hw == 0 ? 1 : hw, 64)));
  {
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&, t]() {
        for (int q = t; q < nsub; q += nth) build_sub(P, q, leaf, small_cap, &subs[q]);
      });
    for (auto& x : th) x.join();
  }
  for (int q = 0; q < nsub; ++q)
    if (!subs[q].err.empty()) {
      set_error("multifrontal plan, subdomain %d: %s", q, subs[q].err.c_str());
      return GDSW_ERR_UNSUPPORTED;
    }
  *M = MfPlan();
  M->leaf = leaf;
  M->sub_sn.assign(nsub + 1, 0);
  M->sub_lv.assign(nsub + 1, 0);
  M->nd_dof.resize(P.sum_m);
  M->nd_loc.resize(P.sum_m);
  M->pullS_ptr.assign(P.sum_m + 1, 0);
  M->sub_stack.assign(nsub + 1, 0);
  int64_t brow = 0, panel = 0;
  for (int q = 0; q < nsub; ++q) {
    const SubMf& R = subs[q];
    const int base = P.om_ptr[q];
    const int sn0 = static_cast<int>(M->sn.size());
    const int nsn = static_cast<int>(R.pos0.size());
    const int64_t panel0 = panel, brow0 = brow;
    M->sub_panel.push_back(panel0);
    M->sub_brow.push_back(static_cast<int>(brow0));
    for (int p = 0; p < R.m; ++p) {
      M->nd_dof[base + p] = P.om_dofs[base + R.perm[p]];
      M->nd_loc[base + p] = static_cast<uint16_t>(R.perm[p]);
    }
    for (int S = 0; S < nsn; ++S) {
      MfSn d;
      d.panel = panel;
      d.pos0 = R.pos0[S];
      d.ns = R.ns[S];
      d.nb = R.nb[S];
      d.uoff = R.uoff[S];
      d.brow = static_cast<int>(brow);
      d.stage = R.stage[S];
      d.nchild = static_cast<int>(R.children[S].size());
      M->sn.push_back(d);
      if (panel - panel0 >= (int64_t(1) << 32) || brow - brow0 >= (int64_t(1) << 32)) {
        set_error("multifrontal plan: subdomain %d too large", q);
        return GDSW_ERR_UNSUPPORTED;
      }
      M->max_nb = std::max(M->max_nb, d.nb);
      M->stack_off.push_back(R.stack_off[S]);
      panel += (panel_entries(R.ns[S], R.nb[S]) + 7) / 8 * 8;   // 16-byte starts for every storage type
      for (int t : R.bset[S]) M->bidx.push_back(static_cast<uint16_t>(t));
      brow += R.nb[S];
    }
    // children (global ids) and the child rows' places in the parent front
    for (int S = 0; S < nsn; ++S) {
      M->ch_ptr.push_back(static_cast<int>(M->ch_list.size()));
      for (int c : R.children[S]) M->ch_list.push_back(sn0 + c);
    }
    M->relF.resize(brow);
    for (int S = 0; S < nsn; ++S)
      for (size_t r = 0; r < R.relF[S].size(); ++r)
        M->relF[M->sn[sn0 + S].brow + r] = static_cast<uint16_t>(R.relF[S][r]);
    // pull lists (the list of a row ends where the next row's begins)
    for (int p = 0; p < R.m; ++p) {
      M->pullS_ptr[base + p] = static_cast<int>(M->pullS_ent.size());
      for (int src : R.pullS[p]) M->pullS_ent.push_back(static_cast<uint16_t>(src));
    }
    for (int S = 0; S < nsn; ++S)
      for (int r = 0; r < R.nb[S]; ++r) {
        M->pullB_ptr.push_back(static_cast<int>(M->pullB_ent.size()));
        for (int src : R.pullB[S][r]) M->pullB_ent.push_back(static_cast<uint16_t>(src));
      }
    // levels: task words (kMfTaskWords each) carry their supernode's layout:
    // panel and first B row relative to the subdomain, pos0 | ns << 16,
    // nb | stage << 16, uoff | (first row or column of the piece) << 16
    auto task = [&](std::vector<uint32_t>& out, int S, int c0) {
      const MfSn& d = M->sn[sn0 + S];
      out.push_back(static_cast<uint32_t>(d.panel - panel0));
      out.push_back(static_cast<uint32_t>(d.brow - brow0));
      out.push_back(uint32_t(d.pos0) | uint32_t(d.ns) << 16);
      out.push_back(uint32_t(d.nb) | uint32_t(d.stage) << 16);
      out.push_back(uint32_t(d.uoff) | uint32_t(c0) << 16);
    };
    const int H = static_cast<int>(R.lev_ptr.size()) - 1;
    for (int l = 0; l < H; ++l) {
      MfLevel L;
      L.rows = static_cast<int>(M->rows.size());
      L.st = static_cast<int>(M->stasks.size() / kMfTaskWords);
      L.xt = static_cast<int>(M->xtasks.size() / kMfTaskWords);
      L.ut = static_cast<int>(M->utasks.size() / kMfTaskWords);
      L.br = static_cast<int>(M->brows.size());
      L.flags = 0;
      for (int k = R.lev_ptr[l]; k < R.lev_ptr[l + 1]; ++k) {
        const int S = R.lev_sn[k];
        if (!R.children[S].empty()) L.flags |= 1;
        for (int i = 0; i < R.ns[S]; ++i) M->rows.push_back(static_cast<uint16_t>(R.pos0[S] + i));
        if (R.small[S]) {
          task(M->stasks, S, 0);
          continue;
        }
        L.flags |= 2;
        for (int i = 0; i < R.ns[S]; ++i) M->brows.push_back(static_cast<uint16_t>(R.pos0[S] + i));
        for (int i = 0; i < R.ns[S]; i += 32) task(M->xtasks, S, i);
        for (int r = 0; r < R.nb[S]; r += 32) task(M->utasks, S, r);
      }
      M->lv.push_back(L);
    }
    // assembly lists
    for (int S = 0; S < nsn; ++S) {
      M->asm_ptr.push_back(static_cast<int>(M->asm_ent.size()));
      for (const auto& a : R.asm_list[S]) {
        M->asm_ent.push_back(a.first);
        M->asm_rc.push_back(a.second);
      }
    }
    M->sub_sn[q + 1] = static_cast<int>(M->sn.size());
    M->sub_lv[q + 1] = static_cast<int>(M->lv.size());
    M->sub_stack[q] = R.stack_peak;
    M->arena_max = std::max(M->arena_max, R.arena);
    M->stage_max = std::max(M->stage_max, R.stage_max);
    M->max_front = std::max(M->max_front, R.max_front);
    M->max_ns = std::max(M->max_ns, R.max_ns);
    M->max_levels = std::max(M->max_levels, H);
  }
  M->pullS_ptr[P.sum_m] = static_cast<int>(M->pullS_ent.size());
  M->pullB_ptr.push_back(static_cast<int>(M->pullB_ent.size()));
  M->ch_ptr.push_back(static_cast<int>(M->ch_list.size()));
  M->asm_ptr.push_back(static_cast<int>(M->asm_ent.size()));
  MfLevel end;
  end.rows = static_cast<int>(M->rows.size());
  end.st = static_cast<int>(M->stasks.size() / kMfTaskWords);
  end.xt = static_cast<int>(M->xtasks.size() / kMfTaskWords);
  end.ut = static_cast<int>(M->utasks.size() / kMfTaskWords);
  end.br = static_cast<int>(M->brows.size());
  end.flags = 0;
  M->lv.push_back(end);
  M->panel_total = panel;
  if (M->pullS_ent.size() + M->pullB_ent.size() >= (size_t(1) << 31) || brow >= (int64_t(1) << 31) ||
      M->asm_ent.size() >= (size_t(1) << 31) || M->rows.size() >= (size_t(1) << 31) ||
      M->xtasks.size() + M->stasks.size() + M->utasks.size() >= (size_t(1) << 31)) {
    set_error("multifrontal plan too large");
    return GDSW_ERR_UNSUPPORTED;
  }
  return GDSW_OK;
}

int64_t mf_work_need(const MfPlan& M, int q) {
  const int64_t f = int64_t(M.max_front) * M.max_front, x = int64_t(M.max_ns) * M.max_ns;
  return (f + x + M.sub_stack[q] + 31) / 32 * 32;
}

int64_t mf_batches(const MfPlan& M, int nsub, std::vector<std::pair<int, int>>* batches) {
  int64_t maxneed = 0;
  for (int q = 0; q < nsub; ++q) maxneed = std::max(maxneed, mf_work_need(M, q));
  const int64_t budget = std::max<int64_t>(maxneed, kMfWorkBudgetBytes / 8);
  int64_t cap = 0;
  if (batches) batches->clear();
  for (int q0 = 0, q1 = 0; q0 < nsub; q0 = q1) {
    int64_t tot = 0;
    while (q1 < nsub && (q1 == q0 || tot + mf_work_need(M, q1) <= budget)) tot += mf_work_need(M, q1++);
    if (batches) batches->push_back({q0, q1});
    cap = std::max(cap, tot);
  }
  return cap;
}

int64_t mf_resident_bytes(const MfPlan& M, int nsub, int64_t sum_m, int64_t pb, int64_t vb) {
  const int64_t brows = static_cast<int64_t>(M.bidx.size());
  return M.panel_total * pb + int64_t(M.sn.size()) * int64_t(sizeof(MfSn)) + int64_t(M.lv.size()) * 16 +
         int64_t(M.rows.size() + M.brows.size()) * 2 +
         int64_t(M.stasks.size() + M.xtasks.size() + M.utasks.size()) * 4 + sum_m * (4 + 2 + 4) + 4 +
         (brows + 1) * 4 + int64_t(M.pullS_ent.size() + M.pullB_ent.size()) * 2 + brows * 2 +
         2 * int64_t(nsub + 1) * 4 + int64_t(nsub) * std::max(1, M.arena_max) * vb;
}

int64_t mf_scratch_bytes(const MfPlan& M, int nsub) {
  return mf_batches(M, nsub, nullptr) * 8 + int64_t(nsub) * 8 +
         int64_t(M.ch_ptr.size() + M.ch_list.size() + M.asm_ptr.size() + M.asm_ent.size() + M.asm_rc.size()) * 4 +
         int64_t(M.relF.size()) * 2 + int64_t(M.stack_off.size()) * 8;
}

}  // namespace gdsw
