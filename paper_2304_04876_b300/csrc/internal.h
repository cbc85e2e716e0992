// Internal declarations of libgdsw: the host-side plan built by the symbolic
// phase, the device context of a handle, and the launchers shared between
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>
#include <memory>
#include <string>
#include <vector>

#include "gdsw.h"

namespace gdsw {

void set_error(const char* fmt, ...);

#define GDSW_CK(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::gdsw::set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                 \
      return GDSW_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

#define GDSW_TRY(expr)            \
  do {                            \
    gdsw_status s_ = (expr);      \
    if (s_ != GDSW_OK) return s_; \
  } while (0)

// ---------------------------------------------------------------------------
// Host plan (symbolic phase, Sec. V-A1 (a)): index structures only, no values.
// ---------------------------------------------------------------------------

// Triangular factor of every subdomain in "level-sliced ELL" form: the rows of
// one level are contiguous, and the off-diagonal entries of a level are stored
// column-major (slot k of row t at off + k*nr + t), padded to the level's
// widest row with a zero entry pointing at the row itself.
struct EllPlan {
  std::vector<int> sub_lev;        // nsub+1: level range of each subdomain
  std::vector<int> lev_start;      // per level: first level-ordered row (absolute)
  std::vector<int> lev_nr;         // rows in the level
  std::vector<int> lev_K;          // padded width
  std::vector<int> lev_off;        // first slot
  std::vector<uint16_t> lrows;     // level-ordered local row index (sum_m)
  std::vector<uint16_t> col;       // local column of each slot
  std::vector<int> src;            // local-CSR entry giving the slot value, -1 = padding
  std::vector<int> dsrc;           // local-CSR diagonal entry of each row, -1 = unit
  int64_t nnz = 0;                 // true entries incl. diagonal
  int64_t slots = 0;
  int max_levels = 0;
};

struct Plan {
  int n = 0, dpn = 1, nnodes = 0, nsub = 0, ncomp = 0;
  int64_t nnz = 0;
  int nb[3] = {1, 1, 1};
  // decomposition (Sec. III)
  std::vector<int> node_sub, node_comp, comp_type;
  std::vector<int> comp_ptr, comp_dofs;   // dofs of each interface component
  std::vector<int> int_ptr, int_dofs;     // interior dofs of each subdomain
  std::vector<int> om_ptr, om_dofs;       // dofs of each overlapping subdomain
  int max_m = 0;
  int64_t sum_m = 0;
  // per dof
  std::vector<int> dof_comp;              // -1 for interior dofs
  std::vector<int> dof_comprow;           // row inside its component
  std::vector<int> dof_introw;            // row inside its subdomain interior
  // local matrices A_s in Omega_s' order, concatenated (rows = sum_m)
  std::vector<int> lm_rowptr;             // sum_m+1, absolute entry offsets
  std::vector<int> lm_col;                // local column
  std::vector<uint16_t> lm_row;           // local row of every entry
  std::vector<int> lm_gent;               // entry of the global CSR
  std::vector<int> lm_tpos;               // entry holding the transposed position
  std::vector<int> lm_diag;               // diagonal entry of each local row
  std::vector<int> lm_sub_ent;            // nsub+1: entry range of each subdomain
  EllPlan L, U;
  // components adjacent (through A) to the interior of each subdomain
  std::vector<std::vector<int>> int_adj;
  std::vector<int> int_bw;                // bandwidth of A_IsIs (local order)
  std::vector<int> om_bw;                 // bandwidth of A_s (local order)
  // scatter lists: per dof, the positions in the concatenated local vectors,
  // ascending subdomain order
  std::vector<int> pull_dof_ptr, pull_dof_pos;
  // coarse-space owners (Sec. III): the components whose coarse columns appear
  // on component c, with the weight of that component in their functions.
  // GDSW: c itself, weight 1; reduced GDSW: the vertices in c's closure, 1/N_c.
  std::vector<int> own_ptr, own_comp;
  std::vector<double> own_w;
  // independent problems of a batch (one problem unless merged)
  int nprob = 1;
  std::vector<int> prob_dof_ptr;          // nprob+1: unknowns of each problem
  std::vector<int> comp_prob;             // problem of each interface component
};

// Coarse-space layout once the rank of every component is known.
// Support of each coarse-space owner: the interface rows its functions cover
// (owner o: entries supp_ptr[o] .. supp_ptr[o+1]).
struct SupportPlan {
  std::vector<int> owners;                // owner components, ascending
  std::vector<int> supp_ptr;              // per owner
  std::vector<int> supp_dof, supp_comp, supp_row;
  std::vector<double> supp_w;
};
gdsw_status build_supports(const Plan& P, SupportPlan* S);

// Rows of one Phi^T r chunk (the kernel stages a chunk's r in shared memory).
constexpr int kPhiChunkRows = 1024;

struct CoarsePlan {
  int n0 = 0;
  std::vector<int> comp_c0;               // first coarse column of each owner component
  std::vector<int> comp_k;                // columns of each owner component (0 for others)
  std::vector<int> supp_colpos;           // per support entry: first column of its owner in the block
  // Phi blocks: b < nsub is the interior of subdomain b, b >= nsub component b-nsub.
  int nblk = 0;
  std::vector<int> brow_ptr, brow_dof;    // every dof exactly once
  std::vector<int> bcol_ptr, bcol;        // coarse columns of each block
  std::vector<int64_t> phi_off;           // column-major block values
  int64_t phi_len = 0;
  std::vector<int> cs_ptr, cs_idx;        // per coarse column: partial slots
  std::vector<int> pull_ptr, pull_pos;    // scatter lists in block-row order
  std::vector<int> dof_blk, dof_blkrow;
  std::vector<int> pos_blk;               // block of every block-row position
  // Phi^T r work split: chunk q covers rows [chunk_r0, chunk_r1) of block
  // chunk_blk; its partial products go to slots chunk_slot[q] .. + block columns
  std::vector<int> chunk_blk, chunk_r0, chunk_r1, chunk_slot;
  int n_cta_chunks = 0;                   // the first n_cta_chunks take a CTA each, the rest a warp
  int n_slots = 0;
  // coarse columns of each problem (A0 is block diagonal over problems)
  std::vector<int> prob_c0;               // nprob+1
};

// Stored width of a level record: levels of width 1-4 are stored row-major
// with each row padded to 4 entries (one vector load of values and one of
// columns per row); wider levels column-major with their own width.
inline int record_width(int K) { return K == 0 ? 0 : (K <= 4 ? 4 : K); }

// Header word 5 of a level record holds its layout (low byte), kRecUpper for
// the records of the second (U) sweep and kRecLevelEnd for the last record of
// a level (the consumers meet at a barrier only there: the rows of one level
// are independent, however many records carry them).
constexpr int kRecUpper = 0x100;
constexpr int kRecLevelEnd = 0x200;

// Largest level record in bytes (a wide level is split into records of at
// most this size).  Every copy into the ring has a fixed cost, so fewer,
// larger records stream faster (measured on B300: 1-4 KB records were 1.2-2.7
// times slower than 32 KB ones).  GDSW_REC_CAP overrides it.
constexpr size_t kRecordCapDefault = 32 * 1024;
inline size_t record_cap() {
  const char* e = getenv("GDSW_REC_CAP");
  const long v = e ? atol(e) : static_cast<long>(kRecordCapDefault);
  return v < 512 ? 512 : static_cast<size_t>(v);
}

// Rows per record when a level of nr rows and width K is split so that one
// record (header, rows, inverse diagonal, values, columns; vb bytes per value)
// stays within `cap` bytes (or holds one node group); a multiple of the node
// group g.
inline int record_piece_rows(int nr, int K, int g, size_t vb, size_t cap) {
  const size_t per_row = 2 + vb + size_t(record_width(K)) * (vb + 2) + size_t(g - 1) * vb;
  size_t rows = cap > 80 + per_row ? (cap - 80) / per_row : 1;
  rows = rows / size_t(g) * size_t(g);
  if (rows < size_t(g)) rows = g;
  return rows >= size_t(nr) ? nr : static_cast<int>(rows);
}

// Multifrontal exact local solver (nested dissection, supernodal fronts, the
// partitioned inverse of each diagonal block).  Positions are ND positions
// inside a subdomain; supernode ids are global (subdomain q owns ids
// sub_sn[q] .. sub_sn[q+1]) and local ones (in rows / task words) are
// relative to sub_sn[q].
struct MfSn {
  int64_t panel;      // first element of [Linv_SS; L_BS], column-major trapezoid:
                      // entry (i, j), i >= j, at panel + j*(ns+nb) - j*(j-1)/2 + (i-j)
  int pos0, ns, nb;   // first ND position, |S|, |B(S)|
  int uoff;           // update vector u_S in the subdomain's arena
  int brow;           // first B row (indexes bidx, pullB_ptr, relF)
  int stage;          // first row of S among the rows of its level
  int nchild;
};
struct MfLevel {
  int rows;           // first entry of the level in rows (ND positions of its unknowns)
  int st, xt, ut;     // first task of the level in stasks / xtasks / utasks
  int br;             // first entry in brows (unknowns of its large supernodes)
  int flags;          // bit 0: some supernode of the level has children;
                      // bit 1: the level has a large supernode
};
// A supernode is small (one warp solves it from a staged copy of its panel)
// when it has at most kMfSmall unknowns, at most kMfSmallNb B rows and its
// panel fits the warp's buffer of mf_buf_bytes(es) bytes, es the solve's value
// size (FP64 solves run 2 CTAs per SM, so their buffers are twice as large).
constexpr int kMfSmall = 32;
constexpr int kMfSmallNb = 128;
constexpr int mf_buf_bytes(int es) { return es == 8 ? 7168 : 3584; }
constexpr int kMfTaskWords = 5;
struct MfPlan {
  int leaf = 0;
  std::vector<MfSn> sn;
  std::vector<int64_t> sub_panel;         // nsub: first panel element of each subdomain
  std::vector<int> sub_brow;              // nsub: first B row of each subdomain
  std::vector<int> sub_sn, sub_lv;        // nsub+1
  std::vector<MfLevel> lv;                // levels of every subdomain, leaves first, plus an end marker
  std::vector<uint16_t> rows;             // per level: ND positions of its unknowns
  std::vector<uint16_t> brows;            // per level: those of its large supernodes, stage order
  // per level, kMfTaskWords per task (see build_mf_plan): small supernodes,
  // 32-row pieces of S and of B(S) of the large ones
  std::vector<uint32_t> stasks, xtasks, utasks;
  std::vector<int> nd_dof;                // sum_m: global unknown of each ND position
  std::vector<uint16_t> nd_loc;           // sum_m: local unknown of each ND position
  std::vector<int> pullS_ptr;             // sum_m+1, into pullS_ent
  std::vector<int> pullB_ptr;             // B rows + 1, into pullB_ent
  std::vector<uint16_t> pullS_ent, pullB_ent;   // arena entries of the children's update vectors
  std::vector<uint16_t> bidx;             // ND position of every B row
  std::vector<uint16_t> relF;             // row of every B row in the parent's front
  std::vector<int> ch_ptr, ch_list;       // children of each supernode (global ids)
  std::vector<int> asm_ptr, asm_ent;      // entries of A_s assembled into each front
  std::vector<uint32_t> asm_rc;           // front row | front column << 16
  std::vector<int64_t> stack_off;         // update matrix of each supernode in its subdomain's stack
  std::vector<int64_t> sub_stack;         // stack doubles of each subdomain
  int64_t panel_total = 0;
  int arena_max = 0, stage_max = 0, max_front = 0, max_ns = 0, max_nb = 0, max_levels = 0;
};
// small_cap: panel entries a warp's staging buffer holds.
gdsw_status build_mf_plan(const Plan& P, int leaf, int small_cap, MfPlan* M);
// Device memory for the fronts, inverse blocks and update stacks of the
// subdomains factored at once.
constexpr int64_t kMfWorkBudgetBytes = int64_t(3) << 30;
// Work doubles of subdomain q's factorisation: front, inverse block, update stack.
int64_t mf_work_need(const MfPlan& M, int q);
// Consecutive subdomain batches whose work fits the budget; returns the
// doubles of the largest batch.
int64_t mf_batches(const MfPlan& M, int nsub, std::vector<std::pair<int, int>>* batches);
// Device bytes the solve keeps (pb bytes per panel value, vb per vector
// value) and the setup's scratch.
int64_t mf_resident_bytes(const MfPlan& M, int nsub, int64_t sum_m, int64_t pb, int64_t vb);
int64_t mf_scratch_bytes(const MfPlan& M, int nsub);
// Nested-dissection leaf size (unknowns); GDSW_MF_LEAF overrides it.
inline int mf_leaf_size() {
  const char* e = getenv("GDSW_MF_LEAF");
  const int v = e ? atoi(e) : 16;
  return v < 1 ? 1 : v;
}

// Device bytes of a handle built from this plan and of the setup's scratch
// (upper bounds; host work only).
gdsw_status estimate_footprint(const Plan& P, const gdsw_csr* A, const gdsw_options& o, int nn, int64_t* resident,
                               int64_t* scratch_peak);
int64_t record_stream_bytes(const Plan& P, int64_t vb, int64_t* nrec);
// Pieces of the node programs (three unknowns per node, FP32): per subdomain,
// sweep (L then U) and level, runs of at most `cap` bytes; each piece's
// subdomain, sweep, level, first node, nodes, widest union of off-node columns
// (K), offset in the stream and bytes.  False when the plan does not take them
// (a level whose rows do not come as whole nodes in solve order, or a node
// wider than a piece).
struct NodePiece { int sub, side, lev, t0, nodes, K; size_t off, bytes; };
// Sliced ELL copy of the global matrix for the SpMV with long rows: slices of
// kSellRows consecutive rows, each as wide as its longest row, entries
// column-major within a slice (entry e of the slice's row r at slice start + e
// * kSellRows + r), columns as 16-bit offsets from the row.  Taken when the mean
// row is longer than 16 entries, every offset fits 16 bits and the padding
// stays under half of the entries; sptr (slices + 1 entry offsets) then holds
// the layout.
constexpr int kSellRows = 8;
bool plan_sell(int n, const int* rowptr, const int* colind, std::vector<int64_t>* sptr);

// The piece limit: kNodePieceBytes, or less by GDSW_NODE_PIECE_BYTES (at least
// 1 KB; several pieces per level, for tests).
size_t node_piece_cap();
bool plan_node_pieces(const Plan& P, size_t cap, std::vector<NodePiece>* pieces, std::vector<int>* pptr,
                      size_t* total, size_t* max_bytes);

gdsw_status build_plan(const gdsw_csr* A, const gdsw_partition* part, const gdsw_options* opt,
                       bool need_levels, Plan* P);
gdsw_status build_coarse_plan(const Plan& P, const SupportPlan& S, const std::vector<int>& comp_rank,
                              bool coarse, CoarsePlan* C);
// Block-diagonal union of independent problems: every index is offset so the
// merged plan describes all problems as one (their subdomains, components and
// levels side by side).
gdsw_status merge_plans(std::vector<Plan>& parts, Plan* out);

// ---------------------------------------------------------------------------
// Device context
// ---------------------------------------------------------------------------

// One triangular factor of all subdomains as the device reads it (see EllPlan).
template <class T>
struct EllDev {
  const int* sub_lev;
  const int4* lev;          // (first row, rows, width, first slot) per level
  const uint16_t* lrows;
  const uint16_t* col;
  const T* val;
  const T* dinv;
  int grp;                  // rows per node, solved in order by one thread
};

// Scalars of the Krylov loop, in device memory.  Reductions write partial sums
// per CTA and the last CTA to finish (ticket counter) adds them in a fixed
// order, so every scalar is bitwise reproducible.
struct KrylovScalars {
  double rz, rz_new, rz_oldz;    // (r,z), new (r,z), (r, z_old) for flexible beta
  double pq, rr, bb;
  double alpha, beta;
  double xalpha;                 // PCG: alpha of the x update still to run (0: none)
  double tol2;                   // tol^2 * ||b||^2
  int iter, done, maxit, flexible;
  int bad;                       // NaN / Inf seen
  int gm_mode;                   // GMRES: 1 = one Gram-Schmidt pass, 2 = a second pass
  unsigned int ticket[8];        // last-block reduction counters
};

constexpr int kNumSMsForCtx = 148;
constexpr int kStepRows = 128;       // rows per step of a row program (= its kernel's threads)
constexpr int kNodePieceBytes = 48 * 1024;   // largest piece of a node program
constexpr int kNodeThreads = 512;            // default threads of the node-program kernel

// Per-problem PCG state of a batched handle.  `start` makes the next
// iteration the PCG prologue for this problem (step lengths 0: r stays, z = M r,
// p = z): 1 for a new right-hand side (||r||^2 of that iteration is ||b||^2 and
// sets the stopping threshold), 2 to continue from a recomputed true residual.
struct BatchScalars {
  double rz, pq, rr, bb, tol2, alpha, beta;
  int iter, done, bad, start;
  int mode;                 // GMRES: 1 one Gram-Schmidt pass this step, 2 a second pass
  int pad;
};

// Per-problem gating of the apply and SpMV kernels of a batched handle: a
// problem whose PCG has stopped (or an idle serving member) costs only this
// check.  `bs` is null on single-problem handles (nothing gated).
struct BatchGate {
  const BatchScalars* bs;
  const int* sub_prob;    // problem of each subdomain
  const int* blk_prob;    // problem of each Phi block
  const int* col_prob;    // problem of each coarse column
  const int* row_ptr;     // nprob+1: unknowns of each problem
  int nprob;
};

#ifdef __CUDACC__
// True when problem p of a batched handle is gated off (it has stopped).
__device__ __forceinline__ bool gate_off(const BatchGate& g, int p) { return g.bs != nullptr && g.bs[p].done; }
__device__ __forceinline__ bool gate_sub_off(const BatchGate& g, int s) {
  return g.bs != nullptr && g.bs[g.sub_prob[s]].done;
}
__device__ __forceinline__ bool gate_blk_off(const BatchGate& g, int b) {
  return g.bs != nullptr && g.bs[g.blk_prob[b]].done;
}
__device__ __forceinline__ bool gate_col_off(const BatchGate& g, int l) {
  return g.bs != nullptr && g.bs[g.col_prob[l]].done;
}
// True when every problem with unknowns in [r0, r1) is gated off.
__device__ __forceinline__ bool gate_rows_off(const BatchGate& g, int r0, int r1) {
  if (g.bs == nullptr) return false;
  int lo = 0, hi = g.nprob - 1;            // last problem whose first unknown <= r0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.row_ptr[mid] <= r0) lo = mid; else hi = mid - 1;
  }
  for (int p = lo; p < g.nprob && g.row_ptr[p] < r1; ++p)
    if (!g.bs[p].done) return false;
  return true;
}
#endif

struct BatchControl {
  unsigned int ndone;
  int all_done;
  int maxit;
  int pad;
  double tol;                     // relative tolerance (thresholds of started problems)
};

// Default bound on a device-side wait: about one second at the B300 SM clock.
constexpr long long kDefaultWaitCycles = 2000000000LL;

struct Ctx {
  int device = 0;
  gdsw_options opt;
  int n = 0, nsub = 0, ncomp = 0, n0 = 0, nblk = 0, dpn = 1;
  int64_t nnz = 0;
  int max_m = 0;
  int64_t sum_m = 0;
  bool fp32 = false;                // preconditioner computes in FP32
  bool fp16 = false;                // level records store the factors in FP16
  bool flexible = false;            // PCG uses the flexible beta (needs (r, z_old))
  std::vector<void*> allocs;
  size_t bytes = 0;
  gdsw_stats stats{};

  // global matrix
  int* rowptr = nullptr;
  int* colind = nullptr;
  double* val = nullptr;
  // overlap
  int* om_ptr = nullptr;
  int* om_dofs = nullptr;
  // level ELL factors (apply precision)
  int* L_sub_lev = nullptr; int4* L_lev = nullptr; uint16_t* L_lrows = nullptr;
  uint16_t* L_col = nullptr; void* L_val = nullptr; void* L_dinv = nullptr;
  int* U_sub_lev = nullptr; int4* U_lev = nullptr; uint16_t* U_lrows = nullptr;
  uint16_t* U_col = nullptr; void* U_val = nullptr; void* U_dinv = nullptr;
  int max_levels = 0;
  // the same factors as a stream of per-level records (pipelined solve)
  uint8_t* rec_stream = nullptr;
  int* rec_ptr = nullptr;            // nsub+1: record range of each subdomain
  uint32_t* rec_off16 = nullptr;     // record offset in 16-byte units
  uint32_t* rec_bytes = nullptr;
  int rec_stage_bytes = 0;
  int64_t rec_total_bytes = 0;
  int rec_stages = 0;                // ring depth chosen at setup (0 = not used)
  int rec_max_width = 0;             // widest level (off-diagonal entries per row)
  // row programs of the prefetching level-scheduled solve (k_local_steps)
  float* step_a = nullptr;           // float4 per row: three entries, inverse diagonal
  uint32_t* step_c = nullptr;        // uint2 per row: three columns, the row
  int2* steps = nullptr;             // {first row, rows | level end << 16}
  int* step_ptr = nullptr;           // nsub+1: step range of each subdomain
  int step_max = 0;                  // most steps of one subdomain
  int step_depth = 0;                // steps in flight per thread; 0: kernel not used
  // node programs of the three-unknowns-per-node solve (k_local_nodes)
  uint8_t* node_stream = nullptr;
  int* node_ptr = nullptr;           // nsub+1: piece range of each subdomain
  int4* node_piece = nullptr;        // {offset / 16, bytes, 0, 0}
  int node_slot_bytes = 0;           // largest piece
  int node_stages = 0;               // ring slots; 0: kernel not used
  int node_threads = 512;            // threads of the node-program kernel (256 or 512)
  // sliced ELL copy for the SpMV with long rows (k_spmv_sell)
  int64_t* sell_ptr = nullptr;
  int16_t* sell_col = nullptr;
  double* sell_val = nullptr;
  int sell_slices = 0;
  int upd_grid = 148;                // CTAs of the PCG residual update (one wave)
  int spmv_sell = 0;                 // 1 / 2: the sliced ELL kernel (4 / 8 in flight) runs the SpMV
  int node_lanes = 4;                // lanes per node of the node-program kernel (2, 4 or 8)
  int rec_tpr = 1;                   // threads per row in the pipelined solve
  int rec_max_rows = 0;              // most rows in one level
  int rec_consumers = 256;           // consumer threads of the pipelined solve
  int rec_prefetch = 0;              // bytes of records kept on their way into L2 ahead of the ring
  bool rec_sf = false;               // pipelined solve without a barrier per level (per-row flags)
  int tri_threads = 256;             // threads of the unpipelined level / Jacobi solve
  // resident Jacobi blocks (see the setup): per subdomain L then U
  uint8_t* jac_stream = nullptr;
  uint32_t* jac_off16 = nullptr;     // 2*nsub: block offsets in 16-byte units
  uint32_t* jac_bytes = nullptr;     // 2*nsub: block sizes
  int jac_max_bytes[2] = {0, 0};     // largest L / U block
  int jac_mode = 0;                  // 0 off, 1 one block resident at a time, 2 the next one arriving meanwhile
  int jac_threads = 1024;            // threads of the resident-block Jacobi kernel (chosen by timing)
  int jac_grid = kNumSMsForCtx;      // its persistent CTAs
  int* derr = nullptr;               // device error flags (bounded waits that ran out)
  long long wait_cycles = 0;         // bound on each device-side wait, SM clock cycles
  int stall_test = 0;                // failure test: one record copy withheld
  // exact local solver, multifrontal (see MfPlan)
  bool mf = false;
  MfSn* mf_sn = nullptr;
  int* mf_sub_sn = nullptr; int* mf_sub_lv = nullptr;
  MfLevel* mf_lv = nullptr;
  uint16_t* mf_rows = nullptr; uint32_t* mf_xt = nullptr; uint32_t* mf_ut = nullptr;
  int* mf_nd_dof = nullptr; uint16_t* mf_nd_loc = nullptr;
  int* mf_pullS_ptr = nullptr; int* mf_pullB_ptr = nullptr;
  uint16_t* mf_pullS = nullptr; uint16_t* mf_pullB = nullptr; uint16_t* mf_bidx = nullptr;
  void* mf_panel = nullptr;
  void* mf_arena_buf = nullptr;      // update vectors, mf_arena entries per subdomain
  std::shared_ptr<const MfPlan> mf_plan_host;   // host plan, kept for gdsw_refactor
  int64_t* mf_sub_panel = nullptr; int* mf_sub_brow = nullptr;
  uint32_t* mf_st = nullptr; uint16_t* mf_brows = nullptr;
  int mf_arena = 0, mf_stage = 0, mf_threads = 256;
  // exact local solver: dense inverses
  void* ainv = nullptr;
  int64_t* ainv_off = nullptr;
  int ainv_chunks = 0;
  // Phi blocks
  int* brow_ptr = nullptr; int* brow_dof = nullptr;
  int* bcol_ptr = nullptr; int* bcol = nullptr;
  int n_bslots = 0;                // entries of bcol (column slots of all Phi blocks)
  void* yslot = nullptr;           // y at every column slot, apply precision
  int64_t* phi_off = nullptr;
  void* phi = nullptr;
  int* cs_ptr = nullptr; int* cs_idx = nullptr;
  int* pull_ptr = nullptr; int* pull_pos = nullptr;
  int* pos_blk = nullptr;
  int* chunk_blk = nullptr; int* chunk_r0 = nullptr; int* chunk_r1 = nullptr; int* chunk_slot = nullptr;
  int n_chunks = 0, n_cta_chunks = 0;
  bool phiT_wide = false;            // Phi^T r: eight columns at a time over a chunk's rows
  int combine_grid = 0;              // resident CTAs of the scatter-add (grid-stride), 4 columns per trip
  int combine_grid8 = 0;             // the same with 8 Phi columns per trip
  int combine_cb = 4;                // Phi columns per trip of the scatter-add (4 or 8)
  int prolong = 0;                   // 1: Phi y formed on the coarse stream (k_prolong) into ubuf
  void* ubuf = nullptr;              // n values of Phi y by block-row position (apply precision)
  int max_bcols = 0;
  int n_slots = 0;
  double* partial = nullptr;     // per (block, column) slot
  double* cvec = nullptr;
  double* yvec = nullptr;
  float* yvec32 = nullptr;           // A0^-1 c rounded once for the FP32 scatter (n0)
  double* A0inv = nullptr;        // one dense block per problem (FP64 apply)
  float* A0inv32 = nullptr;       // the same, rounded once (FP32/FP16 apply)
  float* cvec32 = nullptr;        // c = Phi^T r in FP32 (FP32/FP16 apply)
  int* coarse_prob = nullptr;     // problem of each coarse column
  int* prob_c0 = nullptr;         // coarse column range of each problem
  int64_t* a0_off = nullptr;      // offset of each problem's block
  int coarse_max_block = 0;
  int nprob = 1;
  void* zloc = nullptr;          // local solutions, sum_m
  // Krylov workspace
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b = nullptr;
  double* red = nullptr;         // partial sums for reductions
  int red_len = 0;
  KrylovScalars* ks = nullptr;
  KrylovScalars* ks_host = nullptr;   // pinned mirror
  // GMRES workspace
  double* V = nullptr;           // (restart+1) x n
  double* Zk = nullptr;          // restart x n (right-preconditioned directions)
  double* hcol = nullptr;        // restart+2 doubles
  double* gm = nullptr;          // GMRES state on the device (GmresLayout)
  cudaGraphExec_t gm_exec = nullptr;  // one restart cycle of GMRES
  cudaGraph_t gm_graph = nullptr;
  double gm_keep = 1e-4;         // second Gram-Schmidt pass when ||w - V h||^2 < gm_keep (w, w)
  // graphs
  cudaGraph_t pcg_graph = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaStream_t aux_stream = nullptr;     // coarse branch of the apply
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_x = nullptr, ev_xdone = nullptr;   // PCG x update on the second stream
  // host staging for gdsw_solve_host
  double* hpin = nullptr;
  // events for timed apply
  cudaEvent_t ev[8] = {};
  int red_grid = 0;
  // batched handle (several independent problems)
  int n_tiles = 0;
  double* bgm = nullptr;          // batched GMRES: per-member Hessenberg, rotations, g, coefficients
  double* bgm_y = nullptr;        // per member: 1 / beta at a cycle's start, then y of the cycle
  int* bgm_jd = nullptr;          // per member: Arnoldi steps of the cycle
  int *tile_prob = nullptr, *tile_r0 = nullptr, *tile_r1 = nullptr, *prob_tile_ptr = nullptr;
  std::vector<int> prob_dof_host;
  BatchScalars* bks = nullptr;
  BatchControl* bctl = nullptr;
  cudaGraph_t bgraph = nullptr;
  cudaGraphExec_t bgraph_exec = nullptr;
  cudaGraph_t sgraph = nullptr;          // one batched iteration (continuous batching)
  cudaGraphExec_t sgraph_exec = nullptr;
  BatchScalars* bks_host = nullptr;      // pinned mirror of the per-problem states
  int* sub_prob = nullptr;               // problem of each subdomain (batched handles)
  int* blk_prob = nullptr;               // problem of each Phi block
  int* prob_rows = nullptr;              // nprob+1: unknowns of each problem
  bool serving = false;                  // members started one by one (gdsw_batch_start)
  cudaStream_t bgraph_stream = nullptr;
  int spmv_R = 256, spmv_maxne = 1, spmv_tiles = 1, spmv_grid = kNumSMsForCtx;
  int spmv_U = 8;                      // entries in flight per row in the thread-per-row SpMV
  int16_t* dcol16 = nullptr;           // columns as offsets from the row (when all fit in 16 bits)
  // persistent PCG (k_pcg_persistent): cooperative grid (0: not used), units of
  // 32 local rows per subdomain, grid barrier counter
  int persist_grid = 0;
  size_t persist_smem = 0;
  int* unit_ptr = nullptr;
  int n_units = 0;
  unsigned* pbar = nullptr;
  int spmv_W = 0;                    // lanes per row for long rows (0: the tiled kernel)
  int spmv_pipe = 0;                 // SpMV kernel for short rows (chosen by timing): 0 tiled, 1 tiled with
                                     // the next tile's loads in flight, 2 a thread per row
};

template <class T>
gdsw_status dalloc(Ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return GDSW_ERR_OUT_OF_MEMORY;
  }
  c->allocs.push_back(q);
  c->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return GDSW_OK;
}

template <class T>
gdsw_status upload(Ctx* c, T** p, const std::vector<T>& v, cudaStream_t s) {
  GDSW_TRY(dalloc(c, p, v.size()));
  if (!v.empty())
    GDSW_CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return GDSW_OK;
}

// setup.cu
gdsw_status numeric_setup(Ctx* c, const Plan& P, const gdsw_csr* A, const double* Z, int nn,
                          cudaStream_t s);
// apply.cu
// z = M^-1 r.  When rz_dots is set, the scatter kernel also accumulates
// (r, z_new) and (r, z_old) into the Krylov scalars (z_old read before it is
// overwritten).  Kernels return at once when ks->done is set.
gdsw_status apply_enqueue(Ctx* c, const double* r, double* z, cudaStream_t s, bool rz_dots);
// The apply with every kernel gated on the Krylov stop flag (no dots).
gdsw_status apply_enqueue_gated(Ctx* c, const double* r, double* z, cudaStream_t s);
// The apply of a batched PCG iteration: problems that have stopped are skipped.
gdsw_status apply_enqueue_batch(Ctx* c, const double* r, double* z, cudaStream_t s);
// The gate of the batched handle's iteration (all null on a single problem).
BatchGate batch_gate(const Ctx* c);
gdsw_status apply_timed(Ctx* c, const double* r, double* z, cudaStream_t s, double* ms);
// The PCG form of the apply (dots fused) on one stream, events ev[0..4]
// recorded around its four phases.
gdsw_status apply_timed_dots(Ctx* c, const double* r, double* z, cudaStream_t s, cudaEvent_t* ev);
gdsw_status check_device_errors(Ctx* c, cudaStream_t s);
// multifrontal.cu: the exact local solver for subdomains too large for dense inverses
gdsw_status mf_numeric_setup(Ctx* c, const Plan& P, const double* d_araw, cudaStream_t s);
gdsw_status mf_launch_local(Ctx* c, const double* r, cudaStream_t s, const KrylovScalars* ks);
gdsw_status mf_configure(Ctx* c);
// Largest subdomain (unknowns) whose exact solve uses a dense inverse; larger
// ones use the multifrontal factor.  GDSW_EXACT_DENSE_MAX overrides it.
inline int exact_dense_max() {
  const char* e = getenv("GDSW_EXACT_DENSE_MAX");
  return e ? atoi(e) : 1536;
}
// krylov.cu
gdsw_status krylov_init(Ctx* c, cudaStream_t s);
gdsw_status spmv_enqueue(Ctx* c, const double* x, double* y, cudaStream_t s);
// y = A x on the rows of problems that have not stopped (batched iteration).
gdsw_status spmv_enqueue_batch(Ctx* c, const double* x, double* y, cudaStream_t s);
gdsw_status spmv_configure(Ctx* c, const int* rowptr_host, const int* colind_host, const double* val_host);
gdsw_status persistent_configure(Ctx* c);
gdsw_status pcg_persistent_run(Ctx* c, cudaStream_t s);
gdsw_status solve_pcg(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s);
// One PCG iteration from x = 0 (after its prologue), kernel by kernel on one
// stream with CUDA events: ms[0] SpMV, [1] vector update, [2] local solve,
// [3] Phi^T r, [4] coarse solve, [5] scatter-add (dots fused), [6] direction.
gdsw_status pcg_iteration_timed(Ctx* c, const double* b, cudaStream_t s, double* ms);
gdsw_status solve_gmres(Ctx* c, const double* b, double* x, gdsw_solve_info* info,
                        cudaStream_t s);
// batch.cu
// sub_prob: problem of each subdomain; blk_prob: of each Phi block (subdomain
// interiors, then interface components).
gdsw_status batch_init(Ctx* c, const std::vector<int>& prob_dof_ptr, const std::vector<int>& sub_prob,
                       const std::vector<int>& blk_prob, cudaStream_t s);
gdsw_status solve_pcg_batch(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s);
gdsw_status solve_gmres_batch(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s);
gdsw_status solve_batch(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s);
// Continuous batching on a batched handle: members start, iterate together
// and finish independently (see gdsw_batch_start and the entry points after it).
gdsw_status batch_start(Ctx* c, int member, const double* b, cudaStream_t s);
gdsw_status batch_iterate(Ctx* c, int iterations, cudaStream_t s);
gdsw_status batch_status(Ctx* c, int32_t* done, int32_t* iters, double* relres, cudaStream_t s);
gdsw_status batch_finish(Ctx* c, int member, double* x, gdsw_solve_info* info, int32_t* continued,
                         cudaStream_t s);

constexpr int kNumSMs = 148;

}  // namespace gdsw
