// Device memory a handle will need, from its symbolic plan alone (no device
// work): every array the numeric setup keeps, with the sizes the setup gives
// it, plus the scratch the setup holds on the way.  The coarse space is sized
// as if every owner kept all of its null-space columns, so the figures are
// upper bounds (equal when no column is dropped).
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "internal.h"

namespace gdsw {

namespace {
inline int64_t a16(int64_t x) { return (x + 15) & ~int64_t(15); }
inline int64_t arr(int64_t count, int64_t elem) { return std::max<int64_t>(count, 1) * elem; }
}  // namespace

// Bytes of the per-level record stream of both triangles (the layout the
// numeric setup packs for the pipelined level-scheduled solve).
int64_t record_stream_bytes(const Plan& P, int64_t vb, int64_t* nrec) {
  int64_t total = 0, count = 0;
  for (int q = 0; q < P.nsub; ++q)
    for (int side = 0; side < 2; ++side) {
      const EllPlan& E = side == 0 ? P.L : P.U;
      if (E.sub_lev.empty()) continue;
      for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l) {
        const int K = E.lev_K[l];
        const int piece = record_piece_rows(E.lev_nr[l], K, P.dpn, size_t(vb), record_cap());
        const int64_t Kp = record_width(K);
        for (int t0 = 0; t0 < E.lev_nr[l]; t0 += piece) {
          const int64_t nr = std::min(piece, E.lev_nr[l] - t0);
          total += 32 + a16(2 * nr) + a16(nr * vb) + a16(Kp * nr * vb) + a16(2 * Kp * nr) +
                   (P.dpn > 1 ? a16((int64_t(P.dpn - 1) * nr + 1) * vb) : 0);
          ++count;
        }
      }
    }
  if (nrec) *nrec = count;
  return total;
}

// Bytes of the resident Jacobi blocks (one per subdomain and triangle: header,
// inverse diagonal, values and columns at the subdomain's widest row).
int64_t jacobi_block_bytes(const Plan& P, int64_t vb) {
  int64_t total = 16;
  for (int q = 0; q < P.nsub; ++q) {
    const int64_t m = P.om_ptr[q + 1] - P.om_ptr[q];
    for (int side = 0; side < 2; ++side) {
      const EllPlan& E = side == 0 ? P.L : P.U;
      if (E.sub_lev.empty()) continue;
      int64_t K = 0;
      for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l)
        for (int t = 0; t < E.lev_nr[l]; ++t) {
          int64_t w = 0;
          for (int k = 0; k < E.lev_K[l]; ++k) w += E.src[E.lev_off[l] + int64_t(k) * E.lev_nr[l] + t] >= 0;
          K = std::max(K, w);
        }
      total += 16 + a16(m * vb) + a16(K * m * vb) + a16(2 * K * m);
    }
  }
  return total;
}

bool plan_sell(int n, const int* rowptr, const int* colind, std::vector<int64_t>* sptr) {
  sptr->clear();
  if (n <= 0 || double(rowptr[n]) <= 16.0 * n) return false;
  for (int i = 0; i < n; ++i)
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (colind[e] - i < -32768 || colind[e] - i > 32767) return false;
  const int nsl = (n + kSellRows - 1) / kSellRows;
  sptr->assign(size_t(nsl) + 1, 0);
  for (int q = 0; q < nsl; ++q) {
    int w = 0;
    for (int i = q * kSellRows; i < std::min(n, (q + 1) * kSellRows); ++i) w = std::max(w, rowptr[i + 1] - rowptr[i]);
    (*sptr)[q + 1] = (*sptr)[q] + int64_t(w) * kSellRows;
  }
  if ((*sptr)[nsl] * 2 > int64_t(rowptr[n]) * 3) {
    sptr->clear();
    return false;
  }
  return true;
}

size_t node_piece_cap() {
  size_t cap = kNodePieceBytes;
  if (const char* e = getenv("GDSW_NODE_PIECE_BYTES")) cap = std::min<size_t>(cap, std::max<long>(1024, atol(e)));
  return cap;
}

bool plan_node_pieces(const Plan& P, size_t cap, std::vector<NodePiece>* pieces, std::vector<int>* pptr,
                      size_t* total, size_t* max_bytes) {
  const int nsub = P.nsub;
  pieces->clear();
  pptr->assign(nsub + 1, 0);
  *total = 0;
  *max_bytes = 0;
  for (int q = 0; q < nsub; ++q) {
    for (int side = 0; side < 2; ++side) {
      const EllPlan& E = side == 0 ? P.L : P.U;
      for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l) {
        const int L_nr = E.lev_nr[l];
        if (L_nr % 3 != 0) return false;
        const int nodes = L_nr / 3;
        // the rows of a node consecutive, in solve order (L: 3g, 3g+1, 3g+2; U: reversed)
        for (int t = 0; t < L_nr; ++t) {
          const int g = E.lrows[E.lev_start[l] + t - t % 3] / 3, st = t % 3;
          if (E.lrows[E.lev_start[l] + t] != 3 * g + (side == 0 ? st : 2 - st)) return false;
        }
        // the level's widest union of off-node columns
        int K = 0;
        std::vector<int> u;
        for (int gi = 0; gi < nodes; ++gi) {
          u.clear();
          const int g = E.lrows[E.lev_start[l] + 3 * gi] / 3;
          for (int st = 0; st < 3; ++st)
            for (int k = 0; k < E.lev_K[l]; ++k) {
              const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + 3 * gi + st;
              if (E.src[slot] >= 0 && E.col[slot] / 3 != g) u.push_back(E.col[slot]);
            }
          std::sort(u.begin(), u.end());
          K = std::max<int>(K, static_cast<int>(std::unique(u.begin(), u.end()) - u.begin()));
        }
        // padded to a multiple of 8: chunks of eight columns, of which each of
        // a node's 2, 4 or 8 lanes takes 4, 2 or 1 (vector loads)
        K = (std::max(K, 1) + 7) & ~7;
        // node index, float[8] coefficients, K columns and 3K values per node
        const size_t per_node = 34 + 14 * size_t(K);
        const int cap_nodes = std::max(1, static_cast<int>((cap - 96) / per_node));
        for (int n0 = 0; n0 < nodes; n0 += cap_nodes) {
          const int N = std::min(cap_nodes, nodes - n0);
          const size_t bytes = 16 + size_t(a16(2 * int64_t(N))) + 32 * size_t(N) +
                               size_t(a16(2 * int64_t(N) * K)) + 12 * size_t(N) * K;
          if (bytes > cap) return false;
          pieces->push_back(NodePiece{q, side, l, n0, N, K, *total, bytes});
          *total += size_t(a16(int64_t(bytes)));
          *max_bytes = std::max(*max_bytes, size_t(a16(int64_t(bytes))));
        }
      }
    }
    (*pptr)[q + 1] = static_cast<int>(pieces->size());
  }
  return *total / 4 < (size_t(1) << 31);
}

gdsw_status estimate_footprint(const Plan& P, const gdsw_csr* A, const gdsw_options& o, int nn, int64_t* resident,
                               int64_t* scratch_peak) {
  const bool exact = o.local_solver == GDSW_LOCAL_EXACT;
  const bool low = o.precision != GDSW_PREC_FP64;
  const int64_t v = low ? 4 : 8;                        // apply precision of Phi, inverses, ELL
  const int64_t vrec = o.precision == GDSW_PREC_FP16 ? 2 : v;
  const int64_t n = P.n, nsub = P.nsub, sum_m = P.sum_m, nnz = P.nnz;
  const int64_t nent = static_cast<int64_t>(P.lm_col.size());
  int64_t R = 0, S = 0;

  // matrix, overlap, local solution buffer, device error word
  // (the overlap map padded by four words for the local solve's aligned copies)
  R += arr(n + 1, 4) + arr(nnz, 4) + arr(nnz, 8) + arr(nsub + 1, 4) + arr(sum_m + 4, 4) + arr(sum_m, v) + 4;
  // local matrices and fixed-point sweeps (scratch)
  S += arr(nsub + 1, 4) + arr(sum_m + 1, 4) + 4 * arr(nent, 4) + arr(nent, 2) + arr(sum_m, 8) + 2 * arr(nent, 8);
  if (!exact) {
    S += arr(nent, 4) + 3 * arr(nent, 8) + arr(nent, 4);
    for (const EllPlan* E : {&P.L, &P.U}) {
      R += arr(static_cast<int64_t>(E->sub_lev.size()), 4) + arr(static_cast<int64_t>(E->lev_nr.size()), 16) +
           arr(static_cast<int64_t>(E->lrows.size()), 2) + arr(static_cast<int64_t>(E->col.size()), 2) +
           arr(E->slots, v) + arr(sum_m, v);
      S += arr(static_cast<int64_t>(E->src.size()), 4) + arr(static_cast<int64_t>(E->dsrc.size()), 4);
    }
    int64_t nrec = 0;
    R += arr(record_stream_bytes(P, vrec, &nrec), 1) + arr(nsub + 1, 4) + 2 * arr(nrec, 4);
    if (o.trsv == GDSW_TRSV_JACOBI) R += arr(jacobi_block_bytes(P, vrec), 1) + 2 * arr(2 * nsub, 4);
    // row programs (FP32, one unknown per node, rows of at most 3 entries):
    // 24 bytes per row of each triangle, one int2 per step
    int maxK = 0;
    for (int k : P.L.lev_K) maxK = std::max(maxK, k);
    for (int k : P.U.lev_K) maxK = std::max(maxK, k);
    if (P.dpn == 1 && o.precision == GDSW_PREC_FP32 && o.trsv == GDSW_TRSV_LEVELSCHED && maxK <= 3 && sum_m > 0) {
      int64_t nsteps = 0;
      for (const EllPlan* E : {&P.L, &P.U})
        for (int nr : E->lev_nr) nsteps += (nr + kStepRows - 1) / kStepRows;
      R += arr(2 * sum_m, 16) + arr(2 * sum_m, 8) + arr(nsteps, 8) + arr(nsub + 1, 4);
    }
    // node programs (FP32, three unknowns per node): the stream, piece ranges
    // and table; scratch: value and coefficient positions and sources per sweep
    if (P.dpn == 3 && o.precision == GDSW_PREC_FP32 && o.trsv == GDSW_TRSV_LEVELSCHED && sum_m > 0) {
      std::vector<NodePiece> pcs;
      std::vector<int> pptr;
      size_t total = 0, maxb = 0;
      if (plan_node_pieces(P, node_piece_cap(), &pcs, &pptr, &total, &maxb)) {
        R += arr(static_cast<int64_t>(total) + 16, 1) + arr(nsub + 1, 4) +
             arr(static_cast<int64_t>(pcs.size()), 16);
        for (const EllPlan* E : {&P.L, &P.U}) S += 2 * arr(E->slots, 4) + 2 * arr(sum_m, 4);
      }
    }
  } else if (P.max_m > exact_dense_max() || [&] {
               int64_t d = 0;
               for (int q = 0; q < P.nsub; ++q) d += int64_t(P.om_ptr[q + 1] - P.om_ptr[q]) * (P.om_ptr[q + 1] - P.om_ptr[q]);
               return d > (int64_t(1) << 31);
             }()) {
    // multifrontal exact solver: panels, solve lists, arena; factor work areas
    MfPlan M;
    GDSW_TRY(build_mf_plan(P, mf_leaf_size(), mf_buf_bytes(int(v)) / int(vrec), &M));
    R += mf_resident_bytes(M, P.nsub, sum_m, vrec, v);
    S += mf_scratch_bytes(M, P.nsub);
  } else {
    int64_t dense = 0, band = 0;
    for (int q = 0; q < P.nsub; ++q) {
      const int64_t m = P.om_ptr[q + 1] - P.om_ptr[q];
      dense += m * m;
      band += m * (int64_t(P.om_bw[q]) + 1);
    }
    R += arr(nsub + 1, 8) + arr(dense, v);
    S += arr(dense, 8) + std::min<int64_t>(band * 8, int64_t(4) << 30) + 4 * arr(nsub + 1, 8);
  }

  // coarse space
  const bool coarse = (o.coarse == GDSW_COARSE_GDSW || o.coarse == GDSW_COARSE_RGDSW) && P.ncomp > 0;
  SupportPlan SP;
  GDSW_TRY(build_supports(P, &SP));
  const int nown = static_cast<int>(SP.owners.size());
  const int zcols = nn > 0 ? nn : 1;
  std::vector<int> rank(P.ncomp, 0);
  for (int q = 0; q < nown; ++q)
    rank[SP.owners[q]] = std::min(zcols, SP.supp_ptr[q + 1] - SP.supp_ptr[q]);
  CoarsePlan C;
  GDSW_TRY(build_coarse_plan(P, SP, rank, coarse && nown > 0, &C));
  auto vb = [](const std::vector<int>& x) { return arr(static_cast<int64_t>(x.size()), 4); };
  R += vb(C.brow_ptr) + vb(C.brow_dof) + vb(C.bcol_ptr) + vb(C.bcol) +
       arr(std::max<int64_t>(1, static_cast<int64_t>(C.bcol.size())), v) +
       arr(static_cast<int64_t>(C.phi_off.size()), 8) + vb(C.cs_ptr) + vb(C.cs_idx) + vb(C.pull_ptr) +
       vb(C.pull_pos) + vb(C.pos_blk) + vb(C.chunk_blk) + vb(C.chunk_r0) + vb(C.chunk_r1) + vb(C.chunk_slot) +
       arr(C.n_slots, 8) + 2 * arr(C.n0, 8);
  if (coarse && nown > 0) {
    const int64_t sup = SP.supp_ptr[nown];
    S += arr(n * zcols, 8) + 4 * arr(sup, 4) + arr(sup, 8) + arr(sup * zcols, 8) + arr(nown, 4) +
         2 * arr(sup, 4);
  }
  if (C.n0 > 0) {
    int64_t a0 = 0, maxb = 0, band = 0;
    for (int q = 0; q < P.nprob; ++q) {
      const int64_t nb = C.prob_c0[q + 1] - C.prob_c0[q];
      a0 += nb * nb;
      maxb = std::max(maxb, nb);
    }
    for (int q = 0; q < P.nsub; ++q) band += int64_t(P.int_ptr[q + 1] - P.int_ptr[q]) * (int64_t(P.int_bw[q]) + 1);
    // A0^-1 kept in the apply precision; a low-precision apply builds the FP64
    // inverse in scratch and rounds it once (plus c in FP32)
    R += arr(C.n0, 4) + arr(P.nprob + 1, 4) + arr(P.nprob + 1, 8) + arr(a0, v) + arr(C.phi_len, v) +
         (low ? arr(C.n0, 4) : 0);
    // Phi y by block-row position, formed beside the local solves
    if (C.n0 > 0) R += arr(n, v);
    S += arr(C.phi_len, 8) + arr(a0, 8) + (low ? arr(a0, 8) : 0) + arr((maxb + 63) / 64 * 64 * maxb, 8) +
         std::min<int64_t>(band * 8, int64_t(6) << 30) + 8 * arr(nsub + 1, 8) + 6 * arr(n, 4) + 2 * arr(C.n0, 4);
  }

  // Krylov workspace: six vectors, the reduction buffer, scalars; GMRES basis
  // (reduction buffer: partials of any SpMV grid, at most 32 CTAs per SM)
  R += 6 * arr(n, 8) + arr(2 * (nsub + int64_t(P.ncomp)) + 32 * 148 + 64, 8) + 256;
  // the SpMV's 16-bit column offsets (when they fit), and the sliced ELL copy
  // for long rows (values, offsets, slice starts)
  R += arr(P.nnz, 2);
  {
    std::vector<int64_t> sptr;
    if (plan_sell(P.n, A->rowptr, A->colind, &sptr))
      R += arr(sptr.back(), 8) + arr(sptr.back(), 2) + arr(static_cast<int64_t>(sptr.size()), 8);
  }
  // GMRES: basis and preconditioned directions, its state, and the reduction
  // buffer of its fused dot products (2 restart + 4 partial sums per CTA)
  if (o.krylov == GDSW_KRYLOV_GMRES)
    R += (2 * int64_t(o.restart) + 1) * arr(n, 8) + arr(o.restart + 2, 8) + (int64_t(o.restart) + 2) * 10000 +
         arr((2 * int64_t(o.restart) + 4) * 148 * 8 + 64, 8);
  // batched handles: tiles, per-problem states, the problem of each
  // subdomain, Phi block and unknown range
  if (P.nprob > 1)
    R += 4 * arr(n / 4096 + 2 * P.nprob + 1, 4) + arr(P.nprob, 256) + arr(4 * (n / 4096 + P.nprob) + 64, 8) +
         arr(nsub, 4) + arr(nsub + P.ncomp, 4) + arr(P.nprob + 1, 4);
  // batched GMRES: per member its Hessenberg workspace, y and step count; the
  // partials of an Arnoldi step's dots (restart + 2 per tile)
  if (P.nprob > 1 && o.krylov == GDSW_KRYLOV_GMRES) {
    const int64_t m = std::max(1, o.restart);
    R += arr(P.nprob * ((m + 1) * m + 5 * m + 8), 8) + arr(P.nprob * m, 8) + arr(P.nprob, 4) +
         arr((n / 4096 + P.nprob) * (m + 2) + 64, 8);
  }
  *resident = R;
  *scratch_peak = S;
  return GDSW_OK;
}

}  // namespace gdsw
