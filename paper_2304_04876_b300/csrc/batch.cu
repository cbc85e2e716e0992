// Batched PCG over independent problems merged into one handle.
//
// The merged handle holds the block-diagonal union of the problems (one CSR,
// one set of subdomains, one coarse block per problem), so the SpMV and every
// phase of the preconditioner run as one launch for all problems.  The Krylov
// scalars are per problem: vectors are cut into tiles that never straddle two
// problems, every tile writes its partial dot products, and one warp per
// problem adds its tiles in order (deterministic).  Each problem stops updating
// once it has converged; the iteration runs in a CUDA graph behind a device-side
// while node until every problem has stopped.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gdsw {

namespace {

constexpr int kTileRows = 4096;
constexpr int kThreads = 256;

// Per-member workspace: H ((m+1) x m, row-major), cs, sn (m), g (m+1),
// h1, h2 (m+2: k coefficients and (w, w)), beta (2).
struct BgLayout {
  int m;
  __host__ __device__ explicit BgLayout(int m_) : m(m_) {}
  __host__ __device__ int cs() const { return (m + 1) * m; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int h1() const { return g() + m + 1; }
  __host__ __device__ int h2() const { return h1() + m + 2; }
  __host__ __device__ int beta() const { return h2() + m + 2; }
  __host__ __device__ int total() const { return beta() + 2; }
};


// per-tile partial of (a, b) into part[2 t + slot] (tiles of stopped problems skip)
__global__ void __launch_bounds__(kThreads) k_bdot(const int* __restrict__ tile_prob,
                                                   const int* __restrict__ tile_r0,
                                                   const int* __restrict__ tile_r1,
                                                   const double* __restrict__ a,
                                                   const double* __restrict__ b,
                                                   const BatchScalars* __restrict__ bs,
                                                   double* __restrict__ part, int slot) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  if (bs[tile_prob[t]].done) return;
  double ab = 0.0;
  for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x) ab = fma(a[i], b[i], ab);
  ab = block_sum(ab, sh);
  if (threadIdx.x == 0) part[2 * t + slot] = ab;
}

enum { RED_PQ = 0, RED_RR = 1, RED_RZ = 2 };

// One warp per problem adds its tiles' partials in order and advances the
// problem's PCG state:
//   RED_PQ:   alpha = rz / pq
//   RED_RR:   count the iteration, stop on ||r||^2 <= tol^2 ||b||^2, maxit or breakdown
//   RED_RZ:   beta = (r, z)_new / (r, z)_old, or with `flexible` the
//             flexible beta ((r, z)_new - (r, z_old)) / (r, z)_old
__global__ void k_breduce(int nprob, const int* __restrict__ prob_tile_ptr,
                          const double* __restrict__ part, BatchScalars* bs, int which,
                          BatchControl* ctl, int flexible, cudaGraphConditionalHandle handle,
                          int use_handle) {
  const int lane = threadIdx.x & 31;
  const int pr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pr >= nprob) return;
  BatchScalars& S = bs[pr];
  if (S.done) return;
  double s0 = 0.0, s1 = 0.0;
  for (int t = prob_tile_ptr[pr] + lane; t < prob_tile_ptr[pr + 1]; t += 32) {
    s0 += part[2 * t];
    if (which == RED_RZ && flexible) s1 += part[2 * t + 1];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  if (lane != 0) return;
  if (S.start) {
    // the prologue of a started problem: no step (p = 0), r kept, then
    // z = M r and p = z
    if (which == RED_PQ) {
      S.pq = s0;
      S.alpha = 0.0;
    } else if (which == RED_RR) {
      S.rr = s0;
      if (S.start == 1) {
        S.bb = s0;
        S.tol2 = ctl->tol * ctl->tol * s0;
        if (!isfinite(s0)) { S.bad = 1; S.done = 1; }
        else if (s0 == 0.0) S.done = 1;            // b = 0: x = 0 is the solution
      }
    } else {
      S.beta = 0.0;
      S.rz = s0;
      S.start = 0;
    }
    return;
  }
  if (which == RED_PQ) {
    S.pq = s0;
    S.alpha = S.rz / s0;
    if (!(s0 > 0.0) || !isfinite(S.alpha)) { S.bad = 1; S.alpha = 0.0; }
  } else if (which == RED_RZ) {
    S.beta = (flexible ? s0 - s1 : s0) / S.rz;
    S.rz = s0;
  } else {  // RED_RR
    S.rr = s0;
    S.iter += 1;
    int stop = 0;
    if (S.bad || !isfinite(s0)) { S.bad = 1; stop = 1; }
    else if (s0 <= S.tol2) stop = 1;
    else if (S.iter >= ctl->maxit) stop = 1;
    if (stop) {
      S.done = 1;
      const unsigned int nd = atomicAdd(&ctl->ndone, 1u) + 1;
      if (nd == static_cast<unsigned int>(nprob)) {
        ctl->all_done = 1;
        if (use_handle) cudaGraphSetConditional(handle, 0);
      }
    }
  }
}

// the loop must end even when entered with every problem already stopped
__global__ void k_bguard(BatchControl* ctl, cudaGraphConditionalHandle handle, int use_handle) {
  if (threadIdx.x == 0 && ctl->all_done && use_handle) cudaGraphSetConditional(handle, 0);
}

// x += alpha_p p, r -= alpha_p q; partial ||r||^2 per tile (stopped problems skip)
__global__ void __launch_bounds__(kThreads) k_bupdate(const int* __restrict__ tile_prob,
                                                      const int* __restrict__ tile_r0,
                                                      const int* __restrict__ tile_r1,
                                                      double* __restrict__ x, double* __restrict__ r,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q,
                                                      const BatchScalars* __restrict__ bs,
                                                      double* __restrict__ part) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const BatchScalars& S = bs[tile_prob[t]];
  if (S.done) return;
  const double alpha = S.alpha;
  double rr = 0.0;
  for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) part[2 * t] = rr;
}

// p = z + beta_p p (stopped problems skip); with init, p = z
__global__ void __launch_bounds__(kThreads) k_bpupdate(const int* __restrict__ tile_prob,
                                                       const int* __restrict__ tile_r0,
                                                       const int* __restrict__ tile_r1,
                                                       const double* __restrict__ z,
                                                       double* __restrict__ p,
                                                       const BatchScalars* __restrict__ bs, int init) {
  const int t = blockIdx.x;
  const BatchScalars& S = bs[tile_prob[t]];
  if (S.done) return;
  const double beta = init ? 0.0 : S.beta;
  for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x)
    p[i] = init ? z[i] : fma(beta, p[i], z[i]);
}

// r = b - q
__global__ void k_bresidual(int n, const double* __restrict__ b, const double* __restrict__ q,
                            double* __restrict__ r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] = b[i] - q[i];
}

// Continuous batching: a member's state set for a new right-hand side
// (mode 1) or for a continuation from its true residual (mode 2); every
// member idle (stopped) before the first start.
__global__ void k_bstart(BatchScalars* bs, int member, int mode) {
  BatchScalars& S = bs[member];
  S.start = mode;
  S.done = 0;
  S.bad = 0;
  S.alpha = 0.0;
  S.beta = 0.0;
  if (mode == 1) {
    S.iter = 0;
    S.rz = 1.0;
    S.rr = 0.0;
    S.bb = 0.0;
    S.tol2 = 0.0;
  }
}

__global__ void k_bidle(BatchScalars* bs, int nprob) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nprob; q += gridDim.x * blockDim.x) {
    BatchScalars S = {};
    S.done = 1;
    bs[q] = S;
  }
}

// r = b - A x on rows [row0, row1) (one thread per row, grid-stride), partial
// ||r||^2 per CTA into part[blockIdx.x].
__global__ void __launch_bounds__(kThreads) k_bresid_rows(int row0, int row1, const int* __restrict__ rowptr,
                                                          const int* __restrict__ colind,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ x,
                                                          const double* __restrict__ b, double* __restrict__ r,
                                                          double* __restrict__ part) {
  __shared__ double sh[32];
  double rr = 0.0;
  for (int i = row0 + blockIdx.x * blockDim.x + threadIdx.x; i < row1; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) acc = fma(val[e], x[colind[e]], acc);
    const double ri = b[i] - acc;
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

// The member's true ||r||^2: the partials added in order by one CTA.
__global__ void k_bsum_rr(const double* __restrict__ part, int count, BatchScalars* bs, int member) {
  __shared__ double sh[32];
  const double v = sum_partials(part, count, sh);
  if (threadIdx.x == 0) bs[member].rr = v;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

gdsw_status batch_body(Ctx* c, cudaStream_t s, cudaGraphConditionalHandle h, int use_handle) {
  const int nt = c->n_tiles, np = c->nprob;
  const int rgrid = (np + 7) / 8;
  k_bguard<<<1, 32, 0, s>>>(c->bctl, h, use_handle);
  GDSW_TRY(spmv_enqueue_batch(c, c->p, c->q, s));
  const int flex = c->flexible ? 1 : 0;
  k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->p, c->q, c->bks, c->red, 0);
  k_breduce<<<rgrid, 256, 0, s>>>(np, c->prob_tile_ptr, c->red, c->bks, RED_PQ, c->bctl, flex, h, 0);
  k_bupdate<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->x, c->r, c->p, c->q, c->bks, c->red);
  k_breduce<<<rgrid, 256, 0, s>>>(np, c->prob_tile_ptr, c->red, c->bks, RED_RR, c->bctl, flex, h, use_handle);
  if (flex) k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->z, c->bks, c->red, 1);
  GDSW_TRY(apply_enqueue_batch(c, c->r, c->z, s));
  k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->z, c->bks, c->red, 0);
  k_breduce<<<rgrid, 256, 0, s>>>(np, c->prob_tile_ptr, c->red, c->bks, RED_RZ, c->bctl, flex, h, 0);
  k_bpupdate<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->z, c->p, c->bks, 0);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

}  // namespace

gdsw_status batch_init(Ctx* c, const std::vector<int>& prob_dof_ptr, const std::vector<int>& sub_prob,
                       const std::vector<int>& blk_prob, cudaStream_t s) {
  const int np = static_cast<int>(prob_dof_ptr.size()) - 1;
  GDSW_TRY(upload(c, &c->prob_rows, prob_dof_ptr, s));
  GDSW_TRY(upload(c, &c->sub_prob, sub_prob, s));
  GDSW_TRY(upload(c, &c->blk_prob, blk_prob, s));
  std::vector<int> tp, t0, t1, ptp(np + 1, 0);
  for (int q = 0; q < np; ++q) {
    for (int r0 = prob_dof_ptr[q]; r0 < prob_dof_ptr[q + 1]; r0 += kTileRows) {
      tp.push_back(q);
      t0.push_back(r0);
      t1.push_back(std::min(prob_dof_ptr[q + 1], r0 + kTileRows));
    }
    ptp[q + 1] = static_cast<int>(tp.size());
  }
  c->n_tiles = static_cast<int>(tp.size());
  GDSW_TRY(upload(c, &c->tile_prob, tp, s));
  GDSW_TRY(upload(c, &c->tile_r0, t0, s));
  GDSW_TRY(upload(c, &c->tile_r1, t1, s));
  GDSW_TRY(upload(c, &c->prob_tile_ptr, ptp, s));
  c->prob_dof_host = prob_dof_ptr;
  GDSW_TRY(dalloc(c, &c->bks, np));
  GDSW_TRY(dalloc(c, &c->bctl, 1));
  // partials: the initial residual uses two arrays; batched GMRES one per dot
  // of an Arnoldi step (restart + 2 per tile)
  const int64_t need = c->opt.krylov == GDSW_KRYLOV_GMRES
                           ? std::max<int64_t>(4 * int64_t(c->n_tiles), int64_t(c->n_tiles) * (c->opt.restart + 2))
                           : 4 * int64_t(c->n_tiles);
  if (c->red_len < need + 64) {
    GDSW_TRY(dalloc(c, &c->red, size_t(need) + 64));
    c->red_len = static_cast<int>(need) + 64;
  }
  if (c->opt.krylov == GDSW_KRYLOV_GMRES) {
    const int m = std::max(1, c->opt.restart);
    GDSW_TRY(dalloc(c, &c->bgm, size_t(np) * BgLayout(m).total()));
    GDSW_TRY(dalloc(c, &c->bgm_y, size_t(np) * m));
    GDSW_TRY(dalloc(c, &c->bgm_jd, size_t(np)));
    return GDSW_OK;                                 // the PCG graph is not needed
  }
  const char* env = getenv("GDSW_PCG_GRAPH");
  if (env != nullptr && env[0] == '0') return GDSW_OK;
  GDSW_CK(cudaStreamCreateWithFlags(&c->bgraph_stream, cudaStreamNonBlocking));
  GDSW_CK(cudaGraphCreate(&c->bgraph, 0));
  cudaGraphConditionalHandle h;
  GDSW_CK(cudaGraphConditionalHandleCreate(&h, c->bgraph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams nparams = {};
  nparams.type = cudaGraphNodeTypeConditional;
  nparams.conditional.handle = h;
  nparams.conditional.type = cudaGraphCondTypeWhile;
  nparams.conditional.size = 1;
  cudaGraphNode_t node;
  GDSW_CK(cudaGraphAddNode(&node, c->bgraph, nullptr, nullptr, 0, &nparams));
  cudaGraph_t body = nparams.conditional.phGraph_out[0];
  GDSW_CK(cudaStreamBeginCaptureToGraph(c->bgraph_stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  gdsw_status st = batch_body(c, c->bgraph_stream, h, 1);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->bgraph_stream, &captured);
  if (st != GDSW_OK) return st;
  GDSW_CK(e);
  GDSW_CK(cudaGraphInstantiate(&c->bgraph_exec, c->bgraph, 0));
  return GDSW_OK;
}

// ---- continuous batching ----------------------------------------------------

namespace {

gdsw_status serving_init(Ctx* c, cudaStream_t s) {
  if (c->serving) return GDSW_OK;
  k_bidle<<<(c->nprob + 255) / 256, 256, 0, s>>>(c->bks, c->nprob);
  BatchControl ctl = {};
  ctl.maxit = c->opt.maxit;
  ctl.tol = c->opt.tol;
  GDSW_CK(cudaMemcpyAsync(c->bctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (c->bks_host == nullptr) GDSW_CK(cudaMallocHost(&c->bks_host, sizeof(BatchScalars) * c->nprob));
  const char* env = getenv("GDSW_PCG_GRAPH");
  if (c->sgraph_exec == nullptr && (env == nullptr || env[0] != '0')) {
    // one batched iteration as a graph (no device-side loop: the host admits
    // and retires members between rounds)
    cudaStream_t cs = c->bgraph_stream;
    if (cs == nullptr) {
      GDSW_CK(cudaStreamCreateWithFlags(&c->bgraph_stream, cudaStreamNonBlocking));
      cs = c->bgraph_stream;
    }
    GDSW_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    gdsw_status st = batch_body(c, cs, cudaGraphConditionalHandle{}, 0);
    cudaError_t e = cudaStreamEndCapture(cs, &c->sgraph);
    if (st != GDSW_OK) return st;
    GDSW_CK(e);
    GDSW_CK(cudaGraphInstantiate(&c->sgraph_exec, c->sgraph, 0));
  }
  c->serving = true;
  return GDSW_OK;
}

}  // namespace

gdsw_status batch_start(Ctx* c, int member, const double* b, cudaStream_t s) {
  GDSW_TRY(serving_init(c, s));
  const int off = c->prob_dof_host[member], nm = c->prob_dof_host[member + 1] - off;
  GDSW_CK(cudaMemcpyAsync(c->b + off, b, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->r + off, b, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemsetAsync(c->x + off, 0, sizeof(double) * nm, s));
  GDSW_CK(cudaMemsetAsync(c->p + off, 0, sizeof(double) * nm, s));
  k_bstart<<<1, 1, 0, s>>>(c->bks, member, 1);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

gdsw_status batch_iterate(Ctx* c, int iterations, cudaStream_t s) {
  if (!c->serving) { set_error("gdsw_batch_iterate: no member has been started"); return GDSW_ERR_INVALID_ARG; }
  for (int k = 0; k < iterations; ++k) {
    if (c->sgraph_exec != nullptr) GDSW_CK(cudaGraphLaunch(c->sgraph_exec, s));
    else GDSW_TRY(batch_body(c, s, cudaGraphConditionalHandle{}, 0));
  }
  return GDSW_OK;
}

gdsw_status batch_status(Ctx* c, int32_t* done, int32_t* iters, double* relres, cudaStream_t s) {
  if (!c->serving) GDSW_TRY(serving_init(c, s));
  GDSW_CK(cudaMemcpyAsync(c->bks_host, c->bks, sizeof(BatchScalars) * c->nprob, cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  GDSW_TRY(check_device_errors(c, s));
  for (int q = 0; q < c->nprob; ++q) {
    const BatchScalars& S = c->bks_host[q];
    if (done) done[q] = S.done;
    if (iters) iters[q] = S.iter;
    if (relres) relres[q] = S.bb > 0.0 ? std::sqrt(S.rr / S.bb) : 0.0;
  }
  return GDSW_OK;
}

gdsw_status batch_finish(Ctx* c, int member, double* x, gdsw_solve_info* info, int32_t* continued,
                         cudaStream_t s) {
  if (!c->serving) { set_error("gdsw_batch_finish: no member has been started"); return GDSW_ERR_INVALID_ARG; }
  const int off = c->prob_dof_host[member], nm = c->prob_dof_host[member + 1] - off;
  BatchScalars S;
  GDSW_CK(cudaMemcpyAsync(&S, c->bks + member, sizeof(S), cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (!S.done) { set_error("gdsw_batch_finish: member %d is still iterating", member); return GDSW_ERR_INVALID_ARG; }
  // the true residual r = b - A x of the member, and its norm
  const int grid = std::max(1, std::min(1024, (nm + kThreads - 1) / kThreads));
  k_bresid_rows<<<grid, kThreads, 0, s>>>(off, off + nm, c->rowptr, c->colind, c->val, c->x, c->b, c->r, c->red);
  k_bsum_rr<<<1, 256, 0, s>>>(c->red, grid, c->bks, member);
  GDSW_CK(cudaGetLastError());
  GDSW_CK(cudaMemcpyAsync(&S, c->bks + member, sizeof(S), cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  const bool ok = S.bb == 0.0 || S.rr <= S.tol2;
  const bool give_up = S.bad || S.iter >= c->opt.maxit || !std::isfinite(S.rr);
  if (!ok && !give_up) {
    // continue from the true residual (now in r): p = 0, then the prologue
    GDSW_CK(cudaMemsetAsync(c->p + off, 0, sizeof(double) * nm, s));
    k_bstart<<<1, 1, 0, s>>>(c->bks, member, 2);
    GDSW_CK(cudaGetLastError());
    if (continued) *continued = 1;
    return GDSW_OK;
  }
  if (continued) *continued = 0;
  if (x) GDSW_CK(cudaMemcpyAsync(x, c->x + off, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (info) {
    info->iters = S.iter;
    info->converged = ok ? 1 : 0;
    info->true_relres = S.bb > 0.0 ? std::sqrt(S.rr / S.bb) : 0.0;
    info->seconds = 0.0;
  }
  return GDSW_OK;
}

// Batched PCG: every problem of the merged handle solved at once, each with its
// own alpha, beta and stopping test; info[p] per problem.
gdsw_status solve_pcg_batch(Ctx* c, const double* b, double* x, gdsw_solve_info* info,
                            cudaStream_t s) {
  const double t0 = now_s();
  const int n = c->n, np = c->nprob, nt = c->n_tiles;
  const int rgrid = (np + 7) / 8;
  GDSW_CK(cudaMemcpyAsync(c->b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->x, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  // (a whole-batch solve ends any continuous batching on the handle)
  c->serving = false;
  GDSW_CK(cudaMemsetAsync(c->bks, 0, sizeof(BatchScalars) * np, s));
  BatchControl ctl = {};
  ctl.maxit = c->opt.maxit;
  ctl.tol = c->opt.tol;
  GDSW_CK(cudaMemcpyAsync(c->bctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
  const int vg = std::min(kNumSMs * 8, (n + kThreads - 1) / kThreads);
  // initial residual r = b - A x0, rr and bb per problem
  GDSW_TRY(spmv_enqueue(c, c->x, c->q, s));
  k_bresidual<<<vg, kThreads, 0, s>>>(n, c->b, c->q, c->r);
  k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->b, c->b, c->bks, c->red, 0);
  k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->r, c->bks, c->red + 2 * nt, 0);
  GDSW_CK(cudaGetLastError());
  std::vector<double> part(4 * size_t(nt));
  GDSW_CK(cudaMemcpyAsync(part.data(), c->red, sizeof(double) * 4 * nt, cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  std::vector<int> tile_ptr(np + 1, 0);
  {
    int t = 0;
    for (int q = 0; q < np; ++q) {
      for (int r0 = c->prob_dof_host[q]; r0 < c->prob_dof_host[q + 1]; r0 += kTileRows) ++t;
      tile_ptr[q + 1] = t;
    }
  }
  std::vector<BatchScalars> hs(np);
  std::vector<double> bb(np, 0.0), rr(np, 0.0);
  int ndone = 0;
  for (int q = 0; q < np; ++q) {
    for (int t = tile_ptr[q]; t < tile_ptr[q + 1]; ++t) { bb[q] += part[2 * t]; rr[q] += part[2 * nt + 2 * t]; }
    hs[q] = BatchScalars{};
    hs[q].bb = bb[q];
    hs[q].rr = rr[q];
    hs[q].tol2 = c->opt.tol * c->opt.tol * bb[q];
    hs[q].rz = 1.0;
    if (bb[q] == 0.0 || rr[q] <= hs[q].tol2) { hs[q].done = 1; ++ndone; }
  }
  ctl.ndone = ndone;
  ctl.all_done = ndone == np;
  GDSW_CK(cudaMemcpyAsync(c->bks, hs.data(), sizeof(BatchScalars) * np, cudaMemcpyHostToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->bctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
  std::vector<int> final_iters(np, 0);
  std::vector<double> final_rr(rr);
  for (int round = 0; round < 64 && ndone < np; ++round) {
    // z = M r, (r, z), p = z (first round) or p = z + beta p (continuation)
    const int flex = (c->flexible && round > 0) ? 1 : 0;
    if (flex) k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->z, c->bks, c->red, 1);
    GDSW_TRY(apply_enqueue_batch(c, c->r, c->z, s));
    k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->z, c->bks, c->red, 0);
    k_breduce<<<rgrid, 256, 0, s>>>(np, c->prob_tile_ptr, c->red, c->bks, RED_RZ, c->bctl, flex,
                                    cudaGraphConditionalHandle{}, 0);
    k_bpupdate<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->z, c->p, c->bks, round == 0);
    GDSW_CK(cudaGetLastError());
    if (c->bgraph_exec != nullptr) {
      GDSW_CK(cudaGraphLaunch(c->bgraph_exec, s));
    } else {
      for (;;) {
        GDSW_TRY(batch_body(c, s, cudaGraphConditionalHandle{}, 0));
        BatchControl hc;
        GDSW_CK(cudaMemcpyAsync(&hc, c->bctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
        GDSW_CK(cudaStreamSynchronize(s));
        if (hc.all_done) break;
      }
    }
    // true residual of every problem that stopped on the recurrence
    GDSW_TRY(spmv_enqueue(c, c->x, c->q, s));
    k_bresidual<<<vg, kThreads, 0, s>>>(n, c->b, c->q, c->r);
    GDSW_CK(cudaMemcpyAsync(hs.data(), c->bks, sizeof(BatchScalars) * np, cudaMemcpyDeviceToHost, s));
    GDSW_CK(cudaStreamSynchronize(s));
    // partial (r, r) for all tiles: mark everyone active for the dot, restore after
    std::vector<BatchScalars> act(hs);
    for (auto& v : act) v.done = 0;
    GDSW_CK(cudaMemcpyAsync(c->bks, act.data(), sizeof(BatchScalars) * np, cudaMemcpyHostToDevice, s));
    k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->r, c->bks, c->red, 0);
    GDSW_CK(cudaGetLastError());
    GDSW_CK(cudaMemcpyAsync(part.data(), c->red, sizeof(double) * 2 * nt, cudaMemcpyDeviceToHost, s));
    GDSW_CK(cudaStreamSynchronize(s));
    ndone = 0;
    for (int q = 0; q < np; ++q) {
      double t_rr = 0.0;
      for (int t = tile_ptr[q]; t < tile_ptr[q + 1]; ++t) t_rr += part[2 * t];
      final_rr[q] = t_rr;
      final_iters[q] = hs[q].iter;
      const bool ok = t_rr <= hs[q].tol2 || bb[q] == 0.0;
      const bool give_up = hs[q].bad || hs[q].iter >= c->opt.maxit || !std::isfinite(t_rr);
      if (ok || give_up) { hs[q].done = 1; ++ndone; }
      else hs[q].done = 0;           // continue this problem from its true residual
    }
    ctl.ndone = ndone;
    ctl.all_done = ndone == np;
    GDSW_CK(cudaMemcpyAsync(c->bks, hs.data(), sizeof(BatchScalars) * np, cudaMemcpyHostToDevice, s));
    GDSW_CK(cudaMemcpyAsync(c->bctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
    if (ndone == np) break;
    // continuation: p = z + beta p happens at the top of the next round (round > 0)
  }
  GDSW_CK(cudaMemcpyAsync(x, c->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaStreamSynchronize(s));
  GDSW_TRY(check_device_errors(c, s));
  bool all_ok = true;
  const double el = now_s() - t0;
  for (int q = 0; q < np; ++q) {
    const bool ok = bb[q] == 0.0 || final_rr[q] <= c->opt.tol * c->opt.tol * bb[q];
    all_ok = all_ok && ok;
    if (info) {
      info[q].iters = final_iters[q];
      info[q].converged = ok ? 1 : 0;
      info[q].true_relres = bb[q] == 0.0 ? 0.0 : std::sqrt(final_rr[q] / bb[q]);
      info[q].seconds = el;
    }
  }
  if (!all_ok) { set_error("batched PCG: some problems did not converge"); return GDSW_ERR_NOT_CONVERGED; }
  return GDSW_OK;
}

// ---- batched GMRES(m) --------------------------------------------------------
//
// Restarted right-preconditioned GMRES on every member of a batched handle at
// once (Sec. II's GMRES with the GDSW preconditioner of Eq. 1): the apply and
// the SpMV of an Arnoldi step are one launch for all members (stopped members
// skipped), and the Gram-Schmidt passes run on the member-owned tiles of the
// vectors -- each tile writes its partial (V_i, w), a warp per (member, i) adds
// its tiles in order, one thread per member forms the norm, applies the
// Givens rotations and tests convergence on its own least-squares residual.
// Two Gram-Schmidt passes per step (CGS2), or the single-reduce form with a
// second pass only where the Pythagorean norm cancels.  The host back-solves
// each member's small triangular system after a cycle and adds Z y per member.

namespace {

// V0 = r / beta_p on the tiles of live members
__global__ void __launch_bounds__(kThreads) k_bgm_scale(const int* __restrict__ tile_prob,
                                                        const int* __restrict__ tile_r0,
                                                        const int* __restrict__ tile_r1,
                                                        const double* __restrict__ r,
                                                        const double* __restrict__ inv_beta,
                                                        const BatchScalars* __restrict__ bs, double* __restrict__ v) {
  const int t = blockIdx.x, p = tile_prob[t];
  if (bs[p].done) return;
  const double sc = inv_beta[p];
  for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x) v[i] = r[i] * sc;
}

// partials of (V_i, w), i < k, and (w, w) of one tile into part[t * stride + i]
// (pass 2 only for members whose first pass asked for it)
__global__ void __launch_bounds__(kThreads) k_bgm_dots(int n, int k, const int* __restrict__ tile_prob,
                                                       const int* __restrict__ tile_r0,
                                                       const int* __restrict__ tile_r1,
                                                       const double* __restrict__ V, const double* __restrict__ w,
                                                       const BatchScalars* __restrict__ bs, double* __restrict__ part,
                                                       int stride, int pass) {
  __shared__ double sh[32];
  const int t = blockIdx.x, p = tile_prob[t];
  if (bs[p].done || (pass == 2 && bs[p].mode != 2)) return;
  for (int c0 = 0; c0 <= k; c0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = c0 + u;
        if (col < k) acc[u] = fma(V[int64_t(col) * n + i], wi, acc[u]);
        else if (col == k) acc[u] = fma(wi, wi, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (c0 + u <= k) {
        const double v = block_sum(acc[u], sh);
        if (threadIdx.x == 0) part[int64_t(t) * stride + c0 + u] = v;
      }
    }
  }
}

// h[p][i] = the sum of member p's tile partials of dot i (a warp per (p, i), tiles in order)
__global__ void k_bgm_reduce(int np, int k, const int* __restrict__ prob_tile_ptr,
                             const double* __restrict__ part, int stride, const BatchScalars* __restrict__ bs,
                             double* __restrict__ gm, int m, int pass) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wid >= np * (k + 1)) return;
  const int p = wid / (k + 1), i = wid % (k + 1);
  if (bs[p].done || (pass == 2 && bs[p].mode != 2)) return;
  double v = 0.0;
  for (int t = prob_tile_ptr[p] + lane; t < prob_tile_ptr[p + 1]; t += 32) v += part[int64_t(t) * stride + i];
  v = warp_sum(v);
  const BgLayout L(m);
  if (lane == 0) gm[int64_t(p) * L.total() + (pass == 1 ? L.h1() : L.h2()) + i] = v;
}

// A thread per member.  Pass 1: ||w - V h||^2 = (w, w) - ||h||^2; below `keep`
// of (w, w) (or always, keep > 1) a second pass follows (mode 2).  Pass 2: the
// norm after it.
__global__ void k_bgm_norm(int np, int k, double* __restrict__ gm, int m, BatchScalars* bs, int pass,
                           double keep) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  BatchScalars& S = bs[p];
  if (S.done || (pass == 2 && S.mode != 2)) return;
  const BgLayout L(m);
  double* g = gm + int64_t(p) * L.total();
  const double* h = g + (pass == 1 ? L.h1() : L.h2());
  double sq = 0.0;
  for (int i = 0; i < k; ++i) sq = fma(h[i], h[i], sq);
  const double b2 = h[k] - sq;
  if (pass == 1) {
    if (b2 > keep * h[k]) { S.mode = 1; g[L.beta()] = sqrt(b2); }
    else { S.mode = 2; g[L.beta()] = 0.0; }
  } else {
    g[L.beta() + 1] = b2 > 0.0 ? sqrt(b2) : 0.0;
  }
}

// w -= V h_p on the tiles of live members; the pass that completes the
// orthogonalisation divides by beta (zero beta: left unscaled)
__global__ void __launch_bounds__(kThreads) k_bgm_orth(int n, int k, const int* __restrict__ tile_prob,
                                                       const int* __restrict__ tile_r0,
                                                       const int* __restrict__ tile_r1,
                                                       const double* __restrict__ V, const double* __restrict__ gm,
                                                       int m, const BatchScalars* __restrict__ bs,
                                                       double* __restrict__ w, int pass) {
  const int t = blockIdx.x, p = tile_prob[t];
  const BatchScalars& S = bs[p];
  if (S.done || (pass == 2 && S.mode != 2)) return;
  const bool last = pass == 2 || S.mode == 1;
  const BgLayout L(m);
  const double* g = gm + int64_t(p) * L.total();
  const double* h = g + (pass == 1 ? L.h1() : L.h2());
  const double b = last ? g[L.beta() + pass - 1] : 1.0;
  const double inv = b > 0.0 ? 1.0 / b : 1.0;
  for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < k; ++j) acc = fma(-h[j], V[int64_t(j) * n + i], acc);
    w[i] = last ? acc * inv : acc;
  }
}

// A thread per member: Hessenberg column j, the earlier rotations, the new one,
// and the stopping test on |g_{j+1}| (tolerance, iteration limit, breakdown).
__global__ void k_bgm_givens(int np, int j, int m, double* __restrict__ gm, BatchScalars* bs, int maxit) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  BatchScalars& S = bs[p];
  if (S.done) return;
  const BgLayout L(m);
  double* H = gm + int64_t(p) * L.total();
  double* cs = H + L.cs();
  double* sn = H + L.sn();
  double* g = H + L.g();
  const double* h1 = H + L.h1();
  const double* h2 = H + L.h2();
  const bool two = S.mode == 2;
  for (int i = 0; i <= j; ++i) H[i * m + j] = two ? h1[i] + h2[i] : h1[i];
  const double hn = H[L.beta() + (two ? 1 : 0)];
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = cs[i] * a + sn[i] * b;
    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
  }
  const double d = H[j * m + j];
  const double den = hypot(d, hn);
  if (den == 0.0) { S.bad = 1; S.done = 1; return; }
  cs[j] = d / den;
  sn[j] = hn / den;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  S.iter += 1;
  if (!isfinite(g[j + 1])) S.bad = 1;
  if (!(g[j + 1] * g[j + 1] > S.tol2) || S.iter >= maxit || hn == 0.0 || S.bad) S.done = 1;
}

// x += Z y_p (jd[p] columns) on every tile of a member with steps this cycle
__global__ void __launch_bounds__(kThreads) k_bgm_update_x(int n, const int* __restrict__ tile_prob,
                                                           const int* __restrict__ tile_r0,
                                                           const int* __restrict__ tile_r1,
                                                           const double* __restrict__ Zk,
                                                           const double* __restrict__ yv,
                                                           const int* __restrict__ jd, int m,
                                                           double* __restrict__ x) {
  const int t = blockIdx.x, p = tile_prob[t];
  const int k = jd[p];
  if (k <= 0) return;
  const double* y = yv + int64_t(p) * m;
  for (int i = tile_r0[t] + threadIdx.x; i < tile_r1[t]; i += blockDim.x) {
    double acc = x[i];
    for (int j = 0; j < k; ++j) acc = fma(y[j], Zk[int64_t(j) * n + i], acc);
    x[i] = acc;
  }
}

}  // namespace

gdsw_status solve_gmres_batch(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s) {
  const double t0 = now_s();
  const int n = c->n, np = c->nprob, nt = c->n_tiles;
  const int m = std::max(1, c->opt.restart);
  const BgLayout L(m);
  const int stride = m + 2;
  const double keep = c->opt.gmres_orth == GDSW_GMRES_ORTH_SINGLE ? 1e-4 : 2.0;
  GDSW_CK(cudaMemcpyAsync(c->b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->x, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  c->serving = false;
  const int vg = std::min(kNumSMs * 8, (n + kThreads - 1) / kThreads);
  std::vector<int> tile_ptr(np + 1, 0);
  {
    int t = 0;
    for (int q = 0; q < np; ++q) {
      for (int r0 = c->prob_dof_host[q]; r0 < c->prob_dof_host[q + 1]; r0 += kTileRows) ++t;
      tile_ptr[q + 1] = t;
    }
  }
  std::vector<BatchScalars> hs(np);
  std::vector<double> bb(np, 0.0), rr(np, 0.0), part(4 * size_t(nt));
  std::vector<int> it(np, 0), stalled(np, 0), bad(np, 0), conv(np, 0);
  std::vector<double> gmh(size_t(np) * L.total()), invb(np), yv(size_t(np) * m);
  std::vector<int> jd(np);
  for (int cycle = 0;; ++cycle) {
    // true residual of every member, and ||b||^2 on the first cycle
    for (auto& v : hs) v = BatchScalars{};
    GDSW_CK(cudaMemcpyAsync(c->bks, hs.data(), sizeof(BatchScalars) * np, cudaMemcpyHostToDevice, s));
    GDSW_TRY(spmv_enqueue(c, c->x, c->q, s));
    k_bresidual<<<vg, kThreads, 0, s>>>(n, c->b, c->q, c->r);
    if (cycle == 0)
      k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->b, c->b, c->bks, c->red, 0);
    k_bdot<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->r, c->bks, c->red + 2 * nt, 0);
    GDSW_CK(cudaGetLastError());
    GDSW_CK(cudaMemcpyAsync(part.data(), c->red, sizeof(double) * 4 * nt, cudaMemcpyDeviceToHost, s));
    GDSW_CK(cudaStreamSynchronize(s));
    int nlive = 0;
    for (int q = 0; q < np; ++q) {
      double r2 = 0.0, b2 = 0.0;
      for (int t = tile_ptr[q]; t < tile_ptr[q + 1]; ++t) { r2 += part[2 * nt + 2 * t]; b2 += part[2 * t]; }
      if (cycle == 0) bb[q] = b2;
      rr[q] = r2;
      const double beta = std::sqrt(r2), tolabs = c->opt.tol * std::sqrt(bb[q]);
      conv[q] = bb[q] == 0.0 || beta <= tolabs;
      const bool stop = conv[q] || it[q] >= c->opt.maxit || !std::isfinite(beta) || bad[q] || stalled[q];
      hs[q] = BatchScalars{};
      hs[q].done = stop ? 1 : 0;
      hs[q].iter = it[q];
      hs[q].tol2 = tolabs * tolabs;
      hs[q].mode = 1;
      invb[q] = stop ? 0.0 : 1.0 / beta;
      std::fill(gmh.begin() + int64_t(q) * L.total(), gmh.begin() + int64_t(q + 1) * L.total(), 0.0);
      gmh[int64_t(q) * L.total() + L.g()] = beta;
      nlive += stop ? 0 : 1;
    }
    if (nlive == 0) break;
    GDSW_CK(cudaMemcpyAsync(c->bks, hs.data(), sizeof(BatchScalars) * np, cudaMemcpyHostToDevice, s));
    GDSW_CK(cudaMemcpyAsync(c->bgm, gmh.data(), sizeof(double) * gmh.size(), cudaMemcpyHostToDevice, s));
    GDSW_CK(cudaMemcpyAsync(c->bgm_y, invb.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    k_bgm_scale<<<nt, kThreads, 0, s>>>(c->tile_prob, c->tile_r0, c->tile_r1, c->r, c->bgm_y, c->bks, c->V);
    GDSW_CK(cudaGetLastError());
    const int pg = (np + 255) / 256;
    for (int j = 0; j < m; ++j) {
      const int k = j + 1;
      double* vj = c->V + int64_t(j) * n;
      double* zj = c->Zk + int64_t(j) * n;
      double* w = c->V + int64_t(k) * n;
      GDSW_TRY(apply_enqueue_batch(c, vj, zj, s));
      GDSW_TRY(spmv_enqueue_batch(c, zj, w, s));
      const int rg = (np * (k + 1) + 7) / 8;
      for (int pass = 1; pass <= 2; ++pass) {
        k_bgm_dots<<<nt, kThreads, 0, s>>>(n, k, c->tile_prob, c->tile_r0, c->tile_r1, c->V, w, c->bks, c->red,
                                           stride, pass);
        k_bgm_reduce<<<rg, 256, 0, s>>>(np, k, c->prob_tile_ptr, c->red, stride, c->bks, c->bgm, m, pass);
        k_bgm_norm<<<pg, 256, 0, s>>>(np, k, c->bgm, m, c->bks, pass, keep);
        k_bgm_orth<<<nt, kThreads, 0, s>>>(n, k, c->tile_prob, c->tile_r0, c->tile_r1, c->V, c->bgm, m, c->bks, w,
                                           pass);
      }
      k_bgm_givens<<<pg, 256, 0, s>>>(np, j, m, c->bgm, c->bks, c->opt.maxit);
      GDSW_CK(cudaGetLastError());
    }
    GDSW_CK(cudaMemcpyAsync(gmh.data(), c->bgm, sizeof(double) * gmh.size(), cudaMemcpyDeviceToHost, s));
    std::vector<BatchScalars> after(np);
    GDSW_CK(cudaMemcpyAsync(after.data(), c->bks, sizeof(BatchScalars) * np, cudaMemcpyDeviceToHost, s));
    GDSW_CK(cudaStreamSynchronize(s));
    // y = R^-1 g per member (back substitution), x += Z y
    for (int q = 0; q < np; ++q) {
      jd[q] = 0;
      if (hs[q].done) continue;
      const int steps = after[q].iter - it[q];
      const double* G = gmh.data() + int64_t(q) * L.total();
      double* y = yv.data() + int64_t(q) * m;
      for (int i = steps - 1; i >= 0; --i) {
        double v = G[L.g() + i];
        for (int kk = i + 1; kk < steps; ++kk) v -= G[size_t(i) * m + kk] * y[kk];
        y[i] = v / G[size_t(i) * m + i];
      }
      jd[q] = steps;
      it[q] = after[q].iter;
      bad[q] = after[q].bad;
      stalled[q] = steps == 0;
    }
    GDSW_CK(cudaMemcpyAsync(c->bgm_y, yv.data(), sizeof(double) * yv.size(), cudaMemcpyHostToDevice, s));
    GDSW_CK(cudaMemcpyAsync(c->bgm_jd, jd.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    k_bgm_update_x<<<nt, kThreads, 0, s>>>(n, c->tile_prob, c->tile_r0, c->tile_r1, c->Zk, c->bgm_y, c->bgm_jd, m,
                                           c->x);
    GDSW_CK(cudaGetLastError());
  }
  GDSW_CK(cudaMemcpyAsync(x, c->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaStreamSynchronize(s));
  GDSW_TRY(check_device_errors(c, s));
  bool all_ok = true;
  const double el = now_s() - t0;
  for (int q = 0; q < np; ++q) {
    all_ok = all_ok && conv[q];
    if (info) {
      info[q].iters = it[q];
      info[q].converged = conv[q];
      info[q].true_relres = bb[q] == 0.0 ? 0.0 : std::sqrt(rr[q] / bb[q]);
      info[q].seconds = el;
    }
  }
  if (!all_ok) { set_error("batched GMRES: some problems did not converge"); return GDSW_ERR_NOT_CONVERGED; }
  return GDSW_OK;
}

gdsw_status solve_batch(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s) {
  return c->opt.krylov == GDSW_KRYLOV_GMRES ? solve_gmres_batch(c, b, x, info, s)
                                            : solve_pcg_batch(c, b, x, info, s);
}

}  // namespace gdsw
