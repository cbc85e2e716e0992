// Krylov loops around the preconditioner: CSR SpMV (row tiles for short rows,
// W lanes per row for long ones), fused vector updates with deterministic
// reductions, PCG with its iteration captured in a CUDA graph behind a
// device-side while condition, and right-preconditioned GMRES(m) (Sec. VII)
// with the Arnoldi process, Hessenberg matrix and Givens rotations on the
// device (classical Gram-Schmidt twice, or the single-reduce form).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace gdsw {

namespace {

constexpr int kThreads = 256;
constexpr int kGsThreads = 512;      // threads of the Gram-Schmidt kernels (one CTA per SM)
constexpr int kUpdPairs = 4;         // pairs of the residual update in flight per thread

// y = A x by row tiles of R rows: the tile's values and the gathered x
// entries are loaded once, coalesced, into shared memory, then one thread per
// row forms its sum with one FMA per entry in column order (the FP64 pipe of
// B300 is narrow, so no separate multiply and add).  Every load of a trip is
// issued before any is used (one memory latency for the columns and values,
// one for the gathered x), and the next tile's row pointers are fetched
// before the current tile's sums.  With `ks`, also (x, y) into ks->pq and
// alpha = (r, z) / (x, y) into ks->alpha (the PCG step length, divided once).
template <int R>
__global__ void __launch_bounds__(R) k_spmv_stream(int n, int ntiles, const int* __restrict__ rowptr,
                                                   const int* __restrict__ colind,
                                                   const double* __restrict__ val,
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   double* __restrict__ red, KrylovScalars* ks, BatchGate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int rp[R + 1];
  __shared__ double sh[32];
  if (ks != nullptr && ks->done) return;
  constexpr int U = 8;
  double* va = reinterpret_cast<double*>(smem_raw);
  double dot = 0.0;
  const int t = threadIdx.x;
  // row pointers of the first tile (thread t: row t; thread 0 also the end)
  int tile = blockIdx.x;
  int rp_t = 0, rp_end = 0;
  if (tile < ntiles) {
    const int r0 = tile * R, nr = min(R, n - r0);
    if (t < nr) rp_t = rowptr[r0 + t];
    if (t == 0) rp_end = rowptr[r0 + nr];
  }
  for (; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile * R;
    const int nr = min(R, n - r0);
    if (t < nr) rp[t] = rp_t;
    if (t == 0) rp[nr] = rp_end;
    __syncthreads();
    // (tiles whose problems have all stopped: nothing to load or sum)
    const bool off = gate_rows_off(gate, r0, r0 + nr);
    const int e0 = rp[0];
    const int ne = off ? 0 : rp[nr] - e0;
    double* xa = va + ne;   // gathered x right after the values
    const double* v = val + e0;
    const int* ci = colind + e0;
    for (int j0 = t; j0 < ne; j0 += U * R) {
      int c[U];
      double a[U], xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + u * R;
        c[u] = j < ne ? ci[j] : -1;
        a[u] = j < ne ? v[j] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? x[c[u]] : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + u * R;
        if (j < ne) { va[j] = a[u]; xa[j] = xv[u]; }
      }
    }
    // the next tile's row pointers are in flight during the sums
    const int nt_ = tile + gridDim.x;
    if (nt_ < ntiles) {
      const int q0 = nt_ * R, qn = min(R, n - q0);
      if (t < qn) rp_t = rowptr[q0 + t];
      if (t == 0) rp_end = rowptr[q0 + qn];
    }
    __syncthreads();
    if (t < nr && !off) {
      const int a = rp[t] - e0, b = rp[t + 1] - e0;
      double acc = 0.0;
      for (int q = a; q < b; ++q) acc = fma(va[q], xa[q], acc);
      const int row = r0 + t;
      y[row] = acc;
      dot = fma(x[row], acc, dot);
    }
    __syncthreads();
  }
  if (ks == nullptr) return;
  const double tsum = block_sum(dot, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = tsum;
  if (arrive_last(&ks->ticket[0])) {
    const double s2 = sum_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ks->pq = s2;
      ks->alpha = ks->rz / s2;
    }
  }
}

// The same product with the next tile's columns and values in flight while
// the current tile's sums run: the FP64 pipe (one DFMA per entry) and the
// memory stream overlap within a CTA instead of alternating.  Tiles of R rows
// with at most 8 R entries; row pointers double-buffered in shared memory.
template <int R>
__global__ void __launch_bounds__(R, 2048 / R / 2) k_spmv_pipe(int n, int ntiles, const int* __restrict__ rowptr,
                                                             const int* __restrict__ colind,
                                                             const double* __restrict__ val,
                                                             const double* __restrict__ x, double* __restrict__ y,
                                                             double* __restrict__ red, KrylovScalars* ks,
                                                             BatchGate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int rp[2][R + 1];
  __shared__ double sh[32];
  if (ks != nullptr && ks->done) return;
  constexpr int U = 8;
  double* va = reinterpret_cast<double*>(smem_raw);
  const int t = threadIdx.x;
  double dot = 0.0;
  int tile = blockIdx.x;
  // row pointers of a tile into buffer b
  auto load_rp = [&](int tl, int b) {
    const int r0 = tl * R, nr = min(R, n - r0);
    if (t < nr) rp[b][t] = rowptr[r0 + t];
    if (t == 0) rp[b][nr] = rowptr[r0 + nr];
  };
  if (tile < ntiles) load_rp(tile, 0);
  __syncthreads();
  int c[U];
  double a[U];
  // columns and values of the tile whose row pointers are in buffer b
  auto load_ca = [&](int tl, int b) {
    const int nr = min(R, n - tl * R);
    const int e0 = rp[b][0];
    const int ne = gate_rows_off(gate, tl * R, tl * R + nr) ? 0 : rp[b][nr] - e0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = t + u * R;
      c[u] = j < ne ? colind[e0 + j] : -1;
      a[u] = j < ne ? val[e0 + j] : 0.0;
    }
  };
  if (tile < ntiles) load_ca(tile, 0);
  int buf = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile * R;
    const int nr = min(R, n - r0);
    const bool off = gate_rows_off(gate, r0, r0 + nr);
    const int e0 = rp[buf][0];
    const int ne = off ? 0 : rp[buf][nr] - e0;
    double* xa = va + ne;
    // the gathered x of this tile, then both into shared memory
    double xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? x[c[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = t + u * R;
      if (j < ne) { va[j] = a[u]; xa[j] = xv[u]; }
    }
    const int next = tile + gridDim.x;
    if (next < ntiles) load_rp(next, buf ^ 1);
    __syncthreads();
    // the next tile's columns and values are in flight during the sums
    if (next < ntiles) load_ca(next, buf ^ 1);
    if (t < nr && !off) {
      const int q0 = rp[buf][t] - e0, q1 = rp[buf][t + 1] - e0;
      double acc = 0.0;
      for (int q = q0; q < q1; ++q) acc = fma(va[q], xa[q], acc);
      const int row = r0 + t;
      y[row] = acc;
      dot = fma(x[row], acc, dot);
    }
    __syncthreads();
    buf ^= 1;
  }
  if (ks == nullptr) return;
  const double tsum = block_sum(dot, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = tsum;
  if (arrive_last(&ks->ticket[0])) {
    const double s2 = sum_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ks->pq = s2;
      ks->alpha = ks->rz / s2;
    }
  }
}

// The same product with no shared memory: one thread per row loads its own
// entries (the first U in flight at once, U the longest row within 4..8;
// neighbouring rows' entries are adjacent, so the warp's loads share L1 lines)
// and sums them in column order, so the FP64 FMAs do not queue behind
// shared-memory traffic.
// Column of entry e of row `row`: stored absolute (int) or as a 16-bit offset
// from the row (int16_t: 2 bytes per entry fewer, when every offset fits).
__device__ __forceinline__ int col_of(const int* __restrict__ ci, int e, int) { return ci[e]; }
__device__ __forceinline__ int col_of(const int16_t* __restrict__ ci, int e, int row) { return row + ci[e]; }

template <int U, class CI>
__global__ void __launch_bounds__(256, 4) k_spmv_thread(int n, const int* __restrict__ rowptr,
                                                     const CI* __restrict__ colind,
                                                     const double* __restrict__ val,
                                                     const double* __restrict__ x, double* __restrict__ y,
                                                     double* __restrict__ red, KrylovScalars* ks, BatchGate gate) {
  __shared__ double sh[32];
  if (ks != nullptr && ks->done) return;
  double dot = 0.0;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int row = base + threadIdx.x;
    if (gate_rows_off(gate, base, min(n, base + int(blockDim.x)))) continue;
    if (row < n) {
      const int e0 = rowptr[row], e1 = rowptr[row + 1];
      int c[U];
      double a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        c[u] = e0 + u < e1 ? col_of(colind, e0 + u, row) : -1;
        a[u] = e0 + u < e1 ? val[e0 + u] : 0.0;
      }
      double xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? x[c[u]] : 0.0;
      double acc = 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c[u] >= 0) acc = fma(a[u], xv[u], acc);
      for (int e = e0 + U; e < e1; ++e) acc = fma(val[e], x[col_of(colind, e, row)], acc);
      y[row] = acc;
      dot = fma(x[row], acc, dot);
    }
  }
  if (ks == nullptr) return;
  const double tsum = block_sum(dot, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = tsum;
  if (arrive_last(&ks->ticket[0])) {
    const double s2 = sum_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ks->pq = s2;
      ks->alpha = ks->rz / s2;
    }
  }
}

// y = A x and (x, y) for matrices with long rows: W lanes per row stride over
// its entries (coalesced values and columns), the partial sums meet in a
// shuffle tree of width W; the dot product as in k_spmv_stream.
template <int W>
__global__ void __launch_bounds__(256) k_spmv_rows(int n, const int* __restrict__ rowptr,
                                                   const int* __restrict__ colind,
                                                   const double* __restrict__ val,
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   double* __restrict__ red, KrylovScalars* ks, BatchGate gate) {
  __shared__ double sh[32];
  if (ks != nullptr && ks->done) return;
  const int lane = threadIdx.x % W;
  constexpr int kRows = 256 / W;
  double dot = 0.0;
  for (int base = blockIdx.x * kRows; base < n; base += gridDim.x * kRows) {
    const int row = base + threadIdx.x / W;
    const bool valid = row < n && !gate_rows_off(gate, row, row + 1);
    double acc = 0.0;
    if (valid) {
      const int e1 = rowptr[row + 1];
      for (int e = rowptr[row] + lane; e < e1; e += W) acc = fma(val[e], x[colind[e]], acc);
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, W);
    if (valid && lane == 0) {
      y[row] = acc;
      dot = fma(x[row], acc, dot);
    }
  }
  if (ks == nullptr) return;
  const double t = block_sum(dot, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = t;
  if (arrive_last(&ks->ticket[0])) {
    const double s2 = sum_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ks->pq = s2;
      ks->alpha = ks->rz / s2;
    }
  }
}

// y = A x and (x, y) from the sliced ELL copy (slices of kSellRows = 8 rows,
// entries column-major within a slice, columns as 16-bit offsets from the
// row): a warp per slice, four lanes per row (lane l takes row l % 8 and every
// fourth of its entries from l / 8 on, so the warp reads 32 consecutive
// entries at a time), U entries of a lane in flight, the four partial sums
// added with two shuffles.  Small slices keep the warps' shares even (a 32-row
// slice per warp left most warps idle while a seventh ran a second one); a
// slice's padding entries (value 0, offset 0) cost one DFMA each.  The dot
// product as in k_spmv_stream.
template <int U>
__global__ void __launch_bounds__(256) k_spmv_sell(int n, const int64_t* __restrict__ sptr,
                                                   const int16_t* __restrict__ scol,
                                                   const double* __restrict__ sval,
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   double* __restrict__ red, KrylovScalars* ks, BatchGate gate) {
  static_assert(kSellRows == 8, "four lanes per row of an 8-row slice");
  __shared__ double sh[32];
  if (ks != nullptr && ks->done) return;
  const int lane = threadIdx.x & 31, rr = lane & 7;
  const int nsl = (n + kSellRows - 1) / kSellRows;
  constexpr int kWarps = 256 / 32;
  double dot = 0.0;
  for (int sl = blockIdx.x * kWarps + (threadIdx.x >> 5); sl < nsl; sl += gridDim.x * kWarps) {
    const int row = sl * kSellRows + rr;
    const bool valid = row < n && !gate_rows_off(gate, row, row + 1);
    double acc = 0.0;
    if (valid) {
      const int64_t o1 = sptr[sl + 1];
      int64_t e = sptr[sl] + lane;
      for (; e + (U - 1) * 32 < o1; e += U * 32) {
        int d[U];
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          d[u] = scol[e + u * 32];
          v[u] = sval[e + u * 32];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fma(v[u], x[row + d[u]], acc);
      }
      for (; e < o1; e += 32) acc = fma(sval[e], x[row + scol[e]], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (valid && lane < 8) {
      y[row] = acc;
      dot = fma(x[row], acc, dot);
    }
  }
  if (ks == nullptr) return;
  const double t = block_sum(dot, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = t;
  if (arrive_last(&ks->ticket[0])) {
    const double s2 = sum_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ks->pq = s2;
      ks->alpha = ks->rz / s2;
    }
  }
}

// With alpha = (r,z)/(p,q) (divided once by the SpMV's last CTA): r -= alpha q;
// rr = ||r||^2; then the last CTA counts the iteration, hands alpha to the x
// update (which runs beside the preconditioner: nothing before the next SpMV
// reads x) and decides whether the loop ends.
__global__ void __launch_bounds__(kThreads) k_pcg_update(int n, double* __restrict__ r,
                                                         const double* __restrict__ q,
                                                         double* __restrict__ red, KrylovScalars* ks,
                                                         cudaGraphConditionalHandle handle,
                                                         int use_handle) {
  __shared__ double sh[32];
  if (ks->done) {
    // the loop must end even if it was entered with the flag already set
    if (use_handle && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
    return;
  }
  const double alpha = ks->alpha;
  double rr = 0.0, rr1 = 0.0;
  const int n2 = n >> 1;
  const int stride = gridDim.x * blockDim.x;
  double2* r2 = reinterpret_cast<double2*>(r);
  const double2* q2 = reinterpret_cast<const double2*>(q);
  // kUpdPairs pairs per trip, their loads in flight together and their squares
  // in two accumulators (added at the end)
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUpdPairs - 1) * stride < n2; i += kUpdPairs * stride) {
    double2 qa[kUpdPairs], ra[kUpdPairs];
#pragma unroll
    for (int u = 0; u < kUpdPairs; ++u) {
      qa[u] = q2[i + u * stride];
      ra[u] = r2[i + u * stride];
    }
#pragma unroll
    for (int u = 0; u < kUpdPairs; ++u) {
      ra[u].x = fma(-alpha, qa[u].x, ra[u].x);
      ra[u].y = fma(-alpha, qa[u].y, ra[u].y);
      r2[i + u * stride] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < kUpdPairs; u += 2) {
      rr = fma(ra[u].x, ra[u].x, rr);
      rr = fma(ra[u].y, ra[u].y, rr);
      rr1 = fma(ra[u + 1].x, ra[u + 1].x, rr1);
      rr1 = fma(ra[u + 1].y, ra[u + 1].y, rr1);
    }
  }
  for (; i < n2; i += stride) {
    const double2 qa = q2[i];
    double2 ra = r2[i];
    ra.x = fma(-alpha, qa.x, ra.x);
    ra.y = fma(-alpha, qa.y, ra.y);
    r2[i] = ra;
    rr = fma(ra.x, ra.x, rr);
    rr = fma(ra.y, ra.y, rr);
  }
  rr += rr1;
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int i = n - 1;
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  const double t = block_sum(rr, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = t;
  if (arrive_last(&ks->ticket[1])) {
    const double s = sum_partials(red, gridDim.x, sh);
    if (threadIdx.x == 0) {
      ks->rr = s;
      ks->iter += 1;
      ks->xalpha = alpha;
      int done = 0;
      if (!isfinite(s) || !isfinite(alpha) || !(ks->pq > 0.0)) { ks->bad = 1; done = 1; }
      else if (s <= ks->tol2) done = 1;
      else if (ks->iter >= ks->maxit) done = 1;
      if (done) {
        ks->done = 1;
        if (use_handle) cudaGraphSetConditional(handle, 0);
      }
    }
  }
}

// x += alpha p with the alpha the update kernel handed over (0 when no
// iteration ran since the last x update: nothing to add).  It runs on the
// second stream after the coarse branch and must end before p changes (the
// next k_pupdate waits for it); every CTA reads alpha before it arrives, and
// the last one clears it.
__global__ void __launch_bounds__(kThreads) k_pcg_xupdate(int n, double* __restrict__ x,
                                                          const double* __restrict__ p,
                                                          KrylovScalars* ks) {
  const double alpha = ks->xalpha;
  if (alpha != 0.0) {
    const int n2 = n >> 1;
    double2* x2 = reinterpret_cast<double2*>(x);
    const double2* p2 = reinterpret_cast<const double2*>(p);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
      const double2 pi = p2[i];
      double2 xi = x2[i];
      xi.x = fma(alpha, pi.x, xi.x);
      xi.y = fma(alpha, pi.y, xi.y);
      x2[i] = xi;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) x[n - 1] = fma(alpha, p[n - 1], x[n - 1]);
  }
  if (arrive_last(&ks->ticket[4]) && threadIdx.x == 0) ks->xalpha = 0.0;
}

__global__ void k_pupdate(int n, const double* __restrict__ z, double* __restrict__ p,
                          const KrylovScalars* __restrict__ ks) {
  if (ks->done) return;
  const double beta = ks->beta;
  const int n2 = n >> 1;
  const double2* z2 = reinterpret_cast<const double2*>(z);
  double2* p2 = reinterpret_cast<double2*>(p);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    const double2 zi = z2[i];
    double2 pi = p2[i];
    pi.x = zi.x + beta * pi.x;
    pi.y = zi.y + beta * pi.y;
    p2[i] = pi;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) p[n - 1] = z[n - 1] + beta * p[n - 1];
}

// r = b - q, rr = ||r||^2 and bb = ||b||^2.
__global__ void __launch_bounds__(kThreads) k_residual(int n, const double* __restrict__ b,
                                                       const double* __restrict__ q,
                                                       double* __restrict__ r,
                                                       double* __restrict__ red, KrylovScalars* ks) {
  __shared__ double sh[32];
  double rr = 0.0, bb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = bi - q[i];
    r[i] = ri;
    rr += ri * ri;
    bb += bi * bi;
  }
  const double t1 = block_sum(rr, sh);
  const double t2 = block_sum(bb, sh);
  if (threadIdx.x == 0) { red[2 * blockIdx.x] = t1; red[2 * blockIdx.x + 1] = t2; }
  if (arrive_last(&ks->ticket[3])) {
    double a = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) { a += __ldcg(red + 2 * i); c += __ldcg(red + 2 * i + 1); }
    a = block_sum(a, sh);
    c = block_sum(c, sh);
    if (threadIdx.x == 0) { ks->rr = a; ks->bb = c; }
  }
}

// ---- GMRES helpers -------------------------------------------------------

// h[j] = (V_j, w) for j < k (one CTA row of partials per j), CGS.
// ---- single-reduce GMRES (device-resident Arnoldi and Givens) ----
// Layout of the GMRES state in one device array of doubles (restart m):
// H (m+1) x m row-major | cs m | sn m | g m+1 | h1 m+2 | h2 m+2 | beta 2.
// (with delayed reorthogonalisation: Hraw (m+1) x m the unrotated Hessenberg
// matrix | hp m+1 the new vector's first-pass coefficients | ca m and cc m+1
// the coefficients of the vector update | sc 4 scalars | dt 2m+3 reductions)
struct GmLayout {
  int m;
  __host__ __device__ explicit GmLayout(int m_) : m(m_) {}
  __host__ __device__ int cs() const { return (m + 1) * m; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int h1() const { return g() + m + 1; }
  __host__ __device__ int h2() const { return h1() + m + 2; }
  __host__ __device__ int beta() const { return h2() + m + 2; }
  __host__ __device__ int hraw() const { return beta() + 2; }
  __host__ __device__ int hp() const { return hraw() + (m + 1) * m; }
  __host__ __device__ int ca() const { return hp() + m + 1; }
  __host__ __device__ int cc() const { return ca() + m; }
  __host__ __device__ int sc() const { return cc() + m + 1; }
  __host__ __device__ int dt() const { return sc() + 4; }
  __host__ __device__ int total() const { return dt() + 2 * m + 3; }
};

// ---- GMRES with delayed reorthogonalisation (one reduction per step) ----
//
// The Arnoldi step k applies the operator B = A M^-1 to a vector u_k that is
// orthogonal to the finished basis F = [q_0 .. q_{k-1}] only once.  One fused
// reduction gives a = F^T u_k, (u_k, u_k), F^T w, (u_k, w), (w, w) for w = B u_k.
// From them (one thread): u_k is finished as q_k = (u_k - F a) / sigma, sigma^2
// = (u_k, u_k) - |a|^2 (its second Gram-Schmidt pass, delayed by one step),
// which also finishes Hessenberg column k-1; since B F = Q_{k+1} H (Arnoldi),
// B q_k = (w - Q_{k+1} H a) / sigma, whose projections on Q_{k+1} follow from
// the reduced quantities, and the next vector u_{k+1} = (B q_k - Q_{k+1} h) /
// rho (rho its Pythagorean norm) is formed in the same vector pass that writes
// q_k and M^-1 q_k.  In exact arithmetic this is CGS2 with one reduction per
// step; column k-1 is complete one step later, so the convergence test lags by
// one operator application.

// Step k's scalar work (thread 0 of the reducing CTA): finish u_k and Hessenberg column k-1
// (with its Givens rotation and the residual estimate, which may end the
// cycle), then the coefficients of the vector update.  At the last step of a
// cycle (`final`) only the first part.
__device__ void dc_coef(int k, int m, double* __restrict__ gm, KrylovScalars* ks, int final_step) {
  if (threadIdx.x != 0 || ks->done) return;
  const GmLayout L(m);
  double* H = gm;
  double* cs = gm + L.cs();
  double* sn = gm + L.sn();
  double* g = gm + L.g();
  double* Hr = gm + L.hraw();
  double* hp = gm + L.hp();
  double* ca = gm + L.ca();
  double* cc = gm + L.cc();
  double* sc = gm + L.sc();
  const double* dt = gm + L.dt();
  const double* a = dt;
  const double alpha = final_step ? dt[k] : dt[2 * k];
  double aa = 0.0;
  for (int j = 0; j < k; ++j) aa = fma(a[j], a[j], aa);
  const double s2 = alpha - aa;
  if (!(s2 > 0.0) || !isfinite(s2)) {     // u_k has no new direction: stop the cycle
    if (!isfinite(s2)) ks->bad = 1;
    ks->done = 1;
    return;
  }
  const double sigma = sqrt(s2);
  if (k >= 1) {
    // column k-1: w_{k-1} = Q_k hp + rho u_k = Q_k (hp + rho a) + rho sigma q_k
    const int j = k - 1;
    const double rho = sc[2];
    for (int i = 0; i < k; ++i) Hr[i * m + j] = fma(rho, a[i], hp[i]);
    Hr[k * m + j] = rho * sigma;
    for (int i = 0; i <= j; ++i) H[i * m + j] = Hr[i * m + j];
    const double hn = Hr[k * m + j];
    for (int i = 0; i < j; ++i) {
      const double x0 = H[i * m + j], x1 = H[(i + 1) * m + j];
      H[i * m + j] = cs[i] * x0 + sn[i] * x1;
      H[(i + 1) * m + j] = -sn[i] * x0 + cs[i] * x1;
    }
    const double d = H[j * m + j];
    const double den = hypot(d, hn);
    if (den == 0.0) {
      ks->bad = 1;
      ks->done = 1;
      return;
    }
    cs[j] = d / den;
    sn[j] = hn / den;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    ks->iter += 1;
    if (!isfinite(g[j + 1])) ks->bad = 1;
    if (!(g[j + 1] * g[j + 1] > ks->tol2) || ks->iter >= ks->maxit || ks->bad || hn <= 1e-14 * fabs(den)) {
      ks->done = 1;
      return;
    }
  }
  if (final_step) return;
  // B q_k = (w - Q_{k+1} gv) / sigma with gv = Hr a (columns 0..k-1, rows 0..k);
  // its projections qw / sigma - gv / sigma on Q_{k+1} become hp, and the update
  // u_{k+1} = (w - Q_{k+1} (gv + sigma hp)) / (sigma rho)
  const double* bw = dt + k;
  const double beta = dt[2 * k + 1], gamma = dt[2 * k + 2];
  double ab = 0.0;
  for (int j = 0; j < k; ++j) ab = fma(a[j], bw[j], ab);
  double qg = 0.0, gg = 0.0, hh = 0.0;
  for (int i = 0; i <= k; ++i) {
    double gv = 0.0;
    for (int j = 0; j < k; ++j) gv = fma(Hr[i * m + j], a[j], gv);
    const double qw = i < k ? bw[i] : (beta - ab) / sigma;
    const double h = (qw - gv) / sigma;
    qg = fma(qw, gv, qg);
    gg = fma(gv, gv, gg);
    hh = fma(h, h, hh);
    hp[i] = h;
    cc[i] = fma(sigma, h, gv);
  }
  for (int j = 0; j < k; ++j) ca[j] = a[j];
  const double wt2 = (gamma - 2.0 * qg + gg) / s2;
  const double r2 = wt2 - hh;
  if (!(wt2 >= 0.0) || !isfinite(wt2)) {
    ks->bad = 1;
    ks->done = 1;
    return;
  }
  // (a Pythagorean norm lost to cancellation only scales u_{k+1}; the next
  // step's reorthogonalisation measures its true length)
  const double rho = sqrt(r2 > 1e-28 * wt2 ? r2 : 1e-28 * wt2 + 1e-300);
  sc[0] = 1.0 / sigma;
  sc[1] = 1.0 / (sigma * rho);
  sc[2] = rho;
  sc[3] = sigma;
}

// q_k = (u - F a) / sigma into V_k, M^-1 q_k = (zu - Z_F a) / sigma into Z_k,
// u_{k+1} = (w - Q_{k+1} cc) / (sigma rho) into u (each element read first).
__global__ void __launch_bounds__(kGsThreads, 1) k_dc_update(int n, int k, int m, double* __restrict__ V,
                                                              double* __restrict__ Zk, double* __restrict__ u,
                                                              const double* __restrict__ zu,
                                                              const double* __restrict__ w,
                                                              const double* __restrict__ gm,
                                                              const KrylovScalars* __restrict__ ks) {
  if (ks->done) return;
  const GmLayout L(m);
  const double* ca = gm + L.ca();
  const double* cc = gm + L.cc();
  const double is = gm[L.sc()], isr = gm[L.sc() + 1];
  double* vk = V + int64_t(k) * n;
  double* zk = Zk + int64_t(k) * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double uq = u[i], zz = zu[i], ww = w[i];
    int j = 0;
    // four columns of V and of Z in flight per trip
    for (; j + 4 <= k; j += 4) {
      double vj[4], zj[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        vj[q] = V[int64_t(j + q) * n + i];
        zj[q] = Zk[int64_t(j + q) * n + i];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uq = fma(-ca[j + q], vj[q], uq);
        ww = fma(-cc[j + q], vj[q], ww);
        zz = fma(-ca[j + q], zj[q], zz);
      }
    }
    for (; j < k; ++j) {
      const double vj = V[int64_t(j) * n + i];
      uq = fma(-ca[j], vj, uq);
      ww = fma(-cc[j], vj, ww);
      zz = fma(-ca[j], Zk[int64_t(j) * n + i], zz);
    }
    const double q = uq * is;
    vk[i] = q;
    zk[i] = zz * is;
    ww = fma(-cc[k], q, ww);
    u[i] = ww * isr;
  }
}

// h[j] = the sum of the partials of dot j (one CTA per dot, fixed order).
__global__ void k_gs_reduce(int parts, const double* __restrict__ red, double* __restrict__ h,
                            const KrylovScalars* __restrict__ ks, int need_mode) {
  __shared__ double sh[32];
  if (ks->done || (need_mode != 0 && ks->gm_mode != need_mode)) return;
  const double v = sum_partials(red + int64_t(blockIdx.x) * parts, parts, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = v;
}

// ---- classical Gram-Schmidt of an Arnoldi step (Sec. VII's GMRES) ----
//
// Three launches per step on a grid of one CTA of kGsThreads per SM, each
// CTA a grid-stride share of the rows (FP64: one DFMA per entry, the FP64 pipe and
// the vector stream are the bounds):
//   k_gs_pass1   h1 = [V, w]^T w; the last CTA (ticket) adds the partials in a
//                fixed order and decides on the second pass (mode);
//   k_gs_orth1   w -= V h1, then in mode 2 h2 = [V, w]^T w on the new w (the
//                last CTA adds them), in mode 1 the scaling by 1 / beta and the
//                Givens step (last CTA);
//   k_gs_orth2   mode 2: w -= V h2, scaled by 1 / beta, and the Givens step.
// Every kernel is gated on the stop flag; the mode is uniform over the grid.

// Sums over the 32 lanes of eight values per lane (a[0..7]) as a butterfly
// that halves the values a lane carries at each of the first three steps:
// 4 + 2 + 1 + 1 + 1 adds instead of 8 x 5 (on B300 every FP64 add of a warp
// costs the FP64 pipe as much as a full one).  Afterwards lane l holds the
// warp's sum of column (l >> 2) & 7 in a[0]; fixed order, deterministic.
__device__ __forceinline__ void warp_sum8(double* a) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double mine = b4 ? a[u + 4] : a[u], other = b4 ? a[u] : a[u + 4];
    a[u] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const double mine = b3 ? a[u + 2] : a[u], other = b3 ? a[u] : a[u + 2];
    a[u] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
  }
  {
    const double mine = b2 ? a[1] : a[0], other = b2 ? a[0] : a[1];
    a[0] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
  }
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 2);
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// Partial dots of this CTA's rows for columns c0 .. c0 + NC - 1 of [V_0 ..
// V_{k-1}, x] with x (column k is (x, x)), into red[col * gridDim.x + CTA]:
// per warp the butterfly sums, then the warps' sums in warp order.  Two rows
// per thread per trip keep twice the loads in flight.
template <int NC>
__device__ __forceinline__ void gs_dots_group(int n, int k, int c0, const double* __restrict__ V,
                                              const double* x, double* __restrict__ red, double (*sh)[8]) {
  const double* col[NC];
#pragma unroll
  for (int u = 0; u < NC; ++u) col[u] = c0 + u < k ? V + int64_t(c0 + u) * n : x;
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0;
  const int stride = gridDim.x * blockDim.x;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + stride < n; i += 2 * stride) {
    const double x0 = x[i], x1 = x[i + stride];
    double v0[NC], v1[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      v0[u] = col[u][i];
      v1[u] = col[u][i + stride];
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) acc[u] = fma(v1[u], x1, fma(v0[u], x0, acc[u]));
  }
  if (i < n) {
    const double x0 = x[i];
#pragma unroll
    for (int u = 0; u < NC; ++u) acc[u] = fma(col[u][i], x0, acc[u]);
  }
  warp_sum8(acc);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((lane & 3) == 0) sh[wp][lane >> 2] = acc[0];
  __syncthreads();
  if (threadIdx.x < NC) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += sh[q][threadIdx.x];
    red[int64_t(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
  __syncthreads();
}

// All k + 1 columns, eight at a time (the last group as wide as it needs).
__device__ __forceinline__ void gs_dots(int n, int k, const double* __restrict__ V, const double* x,
                                        double* __restrict__ red, double (*sh)[8]) {
  for (int c0 = 0; c0 <= k; c0 += 8) {
    switch (min(8, k + 1 - c0)) {
      case 1: gs_dots_group<1>(n, k, c0, V, x, red, sh); break;
      case 2: gs_dots_group<2>(n, k, c0, V, x, red, sh); break;
      case 3: gs_dots_group<3>(n, k, c0, V, x, red, sh); break;
      case 4: gs_dots_group<4>(n, k, c0, V, x, red, sh); break;
      case 5: gs_dots_group<5>(n, k, c0, V, x, red, sh); break;
      case 6: gs_dots_group<6>(n, k, c0, V, x, red, sh); break;
      case 7: gs_dots_group<7>(n, k, c0, V, x, red, sh); break;
      default: gs_dots_group<8>(n, k, c0, V, x, red, sh); break;
    }
  }
}

// By the last CTA: h[c] = the CTAs' partials of column c added in CTA order
// (one warp per column), c = 0 .. k; then ||h[0 .. k-1]||^2 by warp 0 (lane
// 0 holds it).  Deterministic whichever CTA is last.
__device__ __forceinline__ double gs_reduce_last(int k, const double* __restrict__ red, double* h) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = gridDim.x;
  for (int cc = wp; cc <= k; cc += nw) {
    double t = 0.0;
    for (int q = lane; q < G; q += 32) t += __ldcg(red + int64_t(cc) * G + q);
    t = warp_sum(t);
    if (lane == 0) h[cc] = t;
  }
  __syncthreads();
  double sq = 0.0;
  if (wp == 0) {
    for (int i = lane; i < k; i += 32) {
      const double hi = h[i];
      sq = fma(hi, hi, sq);
    }
    sq = warp_sum(sq);
  }
  return sq;
}

// w -= V h (k columns) over this CTA's rows; scaled by `inv` when `last`.
// Eight columns' loads in flight per thread.
__device__ __forceinline__ void gs_orth_rows(int n, int k, const double* __restrict__ V, const double* h,
                                             double* w, bool last, double inv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = w[i];
    int j = 0;
    for (; j + 8 <= k; j += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V[int64_t(j + u) * n + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = fma(-h[j + u], v[u], acc);
    }
    for (; j < k; ++j) acc = fma(-h[j], V[int64_t(j) * n + i], acc);
    w[i] = last ? acc * inv : acc;
  }
}

// Column j of the Hessenberg matrix (the coefficients of both passes and
// beta), the earlier rotations applied to it, the new rotation, and the
// least-squares residual |g_{j+1}|, which ends the cycle (and the solve) when
// it is at most tol ||b||, or at maxit, or on breakdown.  Run by the whole
// last CTA: the column and the rotations are staged in shared memory (stage:
// 3m + 4 doubles), one thread rotates, all write the column back.
__device__ void gs_givens(int j, int m, double* __restrict__ gm, KrylovScalars* ks, double* stage) {
  const GmLayout L(m);
  double* H = gm;
  double* cs = gm + L.cs();
  double* sn = gm + L.sn();
  double* g = gm + L.g();
  const double* h1 = gm + L.h1();
  const double* h2 = gm + L.h2();
  __shared__ int ok;
  const bool two = ks->gm_mode == 2;
  double* col = stage;                 // j + 2
  double* cj = stage + (j + 2);        // j
  double* sj = cj + j;                 // j
  for (int i = threadIdx.x; i <= j; i += blockDim.x)
    col[i] = two ? __ldcg(h1 + i) + __ldcg(h2 + i) : __ldcg(h1 + i);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cj[i] = __ldcg(cs + i);
    sj[i] = __ldcg(sn + i);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = __ldcg(gm + L.beta() + (two ? 1 : 0));
    for (int i = 0; i < j; ++i) {
      const double a = col[i], b = col[i + 1];
      col[i] = cj[i] * a + sj[i] * b;
      col[i + 1] = -sj[i] * a + cj[i] * b;
    }
    const double d = col[j];
    const double den = hypot(d, hn);
    ok = den != 0.0;
    if (den == 0.0) {                    // singular: stop, the host sees it as not converged
      ks->bad = 1;
      ks->done = 1;
    } else {
      const double c = d / den, sv = hn / den;
      cs[j] = c;
      sn[j] = sv;
      col[j] = den;
      col[j + 1] = 0.0;
      const double gj = __ldcg(g + j);
      g[j + 1] = -sv * gj;
      g[j] = c * gj;
      ks->iter += 1;
      const double gn = -sv * gj;
      if (!isfinite(gn)) ks->bad = 1;
      if (!(gn * gn > ks->tol2) || ks->iter >= ks->maxit || hn == 0.0 || ks->bad) ks->done = 1;
    }
  }
  __syncthreads();
  if (ok)
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[int64_t(i) * m + j] = col[i];
}

// Pass 1: h1 = V^T w and (w, w) in slot k; the last CTA adds the partials and
// chooses: ||w - V h1||^2 = (w, w) - ||h1||^2 when V is orthonormal; if that
// keeps more than `keep` of (w, w) one pass suffices (mode 1, beta[0] from
// the formula), else a second pass follows (mode 2).  keep > 1 asks for the
// second pass at every step (CGS2).
__global__ void __launch_bounds__(kGsThreads, 1) k_gs_pass1(int n, int k, const double* __restrict__ V,
                                                       const double* __restrict__ w, double* __restrict__ red,
                                                       double* __restrict__ h1, double* __restrict__ beta,
                                                       KrylovScalars* ks, double keep) {
  __shared__ double sh[kGsThreads / 32][8];
  if (ks->done) return;
  gs_dots(n, k, V, w, red, sh);
  if (arrive_last(&ks->ticket[5])) {
    const double sq = gs_reduce_last(k, red, h1);
    if (threadIdx.x == 0) {
      const double ww = h1[k], b2 = ww - sq;
      if (b2 > keep * ww) {
        ks->gm_mode = 1;
        beta[0] = sqrt(b2);
      } else {
        ks->gm_mode = 2;
        beta[0] = 0.0;
      }
    }
  }
}

// w -= V h1; mode 1: scaled by 1 / beta[0] (a zero beta, an exact breakdown,
// leaves w unscaled) and the last CTA takes the Givens step; mode 2: h2 =
// [V, w]^T w on the new w, added up by the last CTA with beta[1] =
// sqrt((w, w) - ||h2||^2).
__global__ void __launch_bounds__(kGsThreads, 1) k_gs_orth1(int n, int k, const double* __restrict__ V,
                                                       const double* __restrict__ h1, double* __restrict__ beta,
                                                       double* __restrict__ w, double* __restrict__ red,
                                                       double* __restrict__ h2, int j, int m, double* gm,
                                                       KrylovScalars* ks) {
  extern __shared__ double stage[];
  __shared__ double sh[kGsThreads / 32][8];
  if (ks->done) return;
  const int mode = ks->gm_mode;
  const double b0 = beta[0];
  gs_orth_rows(n, k, V, h1, w, mode == 1, mode == 1 && b0 > 0.0 ? 1.0 / b0 : 1.0);
  if (mode == 1) {
    if (arrive_last(&ks->ticket[6])) gs_givens(j, m, gm, ks, stage);
    return;
  }
  gs_dots(n, k, V, w, red, sh);
  if (arrive_last(&ks->ticket[6])) {
    const double sq = gs_reduce_last(k, red, h2);
    if (threadIdx.x == 0) {
      const double b2 = h2[k] - sq;
      beta[1] = b2 > 0.0 ? sqrt(b2) : 0.0;
    }
  }
}

// Mode 2: w -= V h2, scaled by 1 / beta[1] (unscaled when zero), and the
// Givens step by the last CTA.
__global__ void __launch_bounds__(kGsThreads, 1) k_gs_orth2(int n, int k, const double* __restrict__ V,
                                                       const double* __restrict__ h2,
                                                       const double* __restrict__ beta, double* __restrict__ w,
                                                       int j, int m, double* gm, KrylovScalars* ks) {
  extern __shared__ double stage[];
  if (ks->done || ks->gm_mode != 2) return;
  const double b1 = beta[1];
  gs_orth_rows(n, k, V, h2, w, true, b1 > 0.0 ? 1.0 / b1 : 1.0);
  if (arrive_last(&ks->ticket[7])) gs_givens(j, m, gm, ks, stage);
}

// ---- delayed reorthogonalisation: the step's reduction in one launch ----

// Partial dots of this CTA's rows for columns c0 .. c0 + NC - 1 of V against u
// (into red rows c0 ..) and, with W, against w (rows k + c0 ..): butterfly warp
// sums, then the warps' sums in warp order.
template <int NC, bool W>
__device__ __forceinline__ void dc_dots_group(int n, int k, int c0, const double* __restrict__ V,
                                              const double* __restrict__ u, const double* __restrict__ w,
                                              double* __restrict__ red, double (*sh)[8], double (*sh2)[8]) {
  const double* col[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) col[q] = V + int64_t(c0 + q) * n;
  double au[8], aw[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    au[q] = 0.0;
    aw[q] = 0.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ui = u[i];
    const double wi = W ? w[i] : 0.0;
    double vv[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) vv[q] = col[q][i];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      au[q] = fma(vv[q], ui, au[q]);
      if (W) aw[q] = fma(vv[q], wi, aw[q]);
    }
  }
  warp_sum8(au);
  if (W) warp_sum8(aw);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((lane & 3) == 0) {
    sh[wp][lane >> 2] = au[0];
    if (W) sh2[wp][lane >> 2] = aw[0];
  }
  __syncthreads();
  if (threadIdx.x < NC) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += sh[q][threadIdx.x];
    red[int64_t(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  } else if (W && threadIdx.x >= 32 && threadIdx.x < 32 + NC) {
    const int cq = threadIdx.x - 32;
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += sh2[q][cq];
    red[int64_t(k + c0 + cq) * gridDim.x + blockIdx.x] = t;
  }
  __syncthreads();
}

template <bool W>
__device__ __forceinline__ void dc_dots(int n, int k, const double* __restrict__ V, const double* __restrict__ u,
                                        const double* __restrict__ w, double* __restrict__ red, double (*sh)[8],
                                        double (*sh2)[8]) {
  for (int c0 = 0; c0 < k; c0 += 8) {
    switch (min(8, k - c0)) {
      case 1: dc_dots_group<1, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      case 2: dc_dots_group<2, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      case 3: dc_dots_group<3, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      case 4: dc_dots_group<4, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      case 5: dc_dots_group<5, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      case 6: dc_dots_group<6, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      case 7: dc_dots_group<7, W>(n, k, c0, V, u, w, red, sh, sh2); break;
      default: dc_dots_group<8, W>(n, k, c0, V, u, w, red, sh, sh2); break;
    }
  }
}

// Step k of the delayed-reorthogonalisation cycle: the partial sums of (V_j,
// u), (V_j, w) for j < k and of (u, u), (u, w), (w, w) (without w only
// (V_j, u) and (u, u)); the last CTA adds them in CTA order into the dots
// array and takes the step's scalar work (dc_coef).  One launch in place of a
// dot, a reduction and a scalar kernel.
__global__ void __launch_bounds__(kGsThreads, 1) k_dc_step(int n, int k, int m, const double* __restrict__ V,
                                                           const double* __restrict__ u,
                                                           const double* __restrict__ w, double* __restrict__ red,
                                                           double* __restrict__ gm, KrylovScalars* ks,
                                                           int final_step) {
  __shared__ double sh[kGsThreads / 32][8], sh2[kGsThreads / 32][8];
  if (ks->done) return;
  const bool W = w != nullptr;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // (u, u), (u, w), (w, w)
  {
    double uu = 0.0, uw = 0.0, ww = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double ui = u[i];
      uu = fma(ui, ui, uu);
      if (W) {
        const double wi = w[i];
        uw = fma(ui, wi, uw);
        ww = fma(wi, wi, ww);
      }
    }
    uu = warp_sum(uu);
    if (W) {
      uw = warp_sum(uw);
      ww = warp_sum(ww);
    }
    if (lane == 0) {
      sh[wp][0] = uu;
      sh[wp][1] = uw;
      sh[wp][2] = ww;
    }
    __syncthreads();
    if (threadIdx.x < (W ? 3 : 1)) {
      double t = 0.0;
      for (int q = 0; q < nw; ++q) t += sh[q][threadIdx.x];
      const int row = W ? 2 * k + threadIdx.x : k;
      red[int64_t(row) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
  if (W) dc_dots<true>(n, k, V, u, w, red, sh, sh2);
  else dc_dots<false>(n, k, V, u, w, red, sh, sh2);
  if (arrive_last(&ks->ticket[5])) {
    const GmLayout L(m);
    double* dt = gm + L.dt();
    const int nd = W ? 2 * k + 3 : k + 1;
    const int G = gridDim.x;
    for (int cc = wp; cc < nd; cc += nw) {
      double t = 0.0;
      for (int q = lane; q < G; q += 32) t += __ldcg(red + int64_t(cc) * G + q);
      t = warp_sum(t);
      if (lane == 0) dt[cc] = t;
    }
    __syncthreads();
    dc_coef(k, m, gm, ks, final_step);
  }
}

// b = a * (*scal); a and b may be the same vector
__global__ void k_scale_copy(int n, const double* a, const double* __restrict__ scal, double* b) {
  const double sc = *scal;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i] * sc;
}

// x += Z y (k columns)
__global__ void k_update_x(int n, int k, const double* __restrict__ Zk, const double* __restrict__ yv,
                           double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int j = 0; j < k; ++j) acc += yv[j] * Zk[int64_t(j) * n + i];
    x[i] = acc;
  }
}

gdsw_status launch_spmv(Ctx* c, const double* x, double* y, cudaStream_t s, KrylovScalars* ks,
                        const BatchGate& gate = BatchGate{}) {
  if (c->spmv_sell) {
    const int grid = std::max(1, std::min(c->spmv_grid, (c->sell_slices + 7) / 8));
    if (c->spmv_sell == 2)
      k_spmv_sell<8><<<grid, 256, 0, s>>>(c->n, c->sell_ptr, c->sell_col, c->sell_val, x, y, c->red, ks, gate);
    else
      k_spmv_sell<4><<<grid, 256, 0, s>>>(c->n, c->sell_ptr, c->sell_col, c->sell_val, x, y, c->red, ks, gate);
    GDSW_CK(cudaGetLastError());
    return GDSW_OK;
  }
  if (c->spmv_W > 0) {
    const int grid = std::max(1, std::min(c->spmv_grid, (c->n + 256 / c->spmv_W - 1) / (256 / c->spmv_W)));
    switch (c->spmv_W) {
      case 4: k_spmv_rows<4><<<grid, 256, 0, s>>>(c->n, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
      case 8: k_spmv_rows<8><<<grid, 256, 0, s>>>(c->n, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
      case 16: k_spmv_rows<16><<<grid, 256, 0, s>>>(c->n, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
      default: k_spmv_rows<32><<<grid, 256, 0, s>>>(c->n, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
    }
    GDSW_CK(cudaGetLastError());
    return GDSW_OK;
  }
  if (c->spmv_pipe == 2) {
    const int grid = std::max(1, std::min(c->spmv_grid, (c->n + 255) / 256));
    switch (c->spmv_U) {
#define GDSW_SPMV_T(UU)                                                                                    \
  case UU:                                                                                                 \
    if (c->dcol16 != nullptr)                                                                              \
      k_spmv_thread<UU, int16_t><<<grid, 256, 0, s>>>(c->n, c->rowptr, c->dcol16, c->val, x, y, c->red, ks, gate); \
    else                                                                                                   \
      k_spmv_thread<UU, int><<<grid, 256, 0, s>>>(c->n, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); \
    break;
      GDSW_SPMV_T(4)
      GDSW_SPMV_T(5)
      GDSW_SPMV_T(6)
      GDSW_SPMV_T(7)
      default: GDSW_SPMV_T(8)
#undef GDSW_SPMV_T
    }
    GDSW_CK(cudaGetLastError());
    return GDSW_OK;
  }
  const int grid = std::min(c->spmv_grid, c->spmv_tiles);
  const size_t shm = size_t(c->spmv_maxne) * 2 * sizeof(double);
  if (c->spmv_pipe) {
    switch (c->spmv_R) {
      case 256: k_spmv_pipe<256><<<grid, 256, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
      case 128: k_spmv_pipe<128><<<grid, 128, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
      case 64: k_spmv_pipe<64><<<grid, 64, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
      default: k_spmv_pipe<32><<<grid, 32, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
    }
    GDSW_CK(cudaGetLastError());
    return GDSW_OK;
  }
  switch (c->spmv_R) {
    case 256: k_spmv_stream<256><<<grid, 256, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
    case 128: k_spmv_stream<128><<<grid, 128, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
    case 64: k_spmv_stream<64><<<grid, 64, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
    default: k_spmv_stream<32><<<grid, 32, shm, s>>>(c->n, c->spmv_tiles, c->rowptr, c->colind, c->val, x, y, c->red, ks, gate); break;
  }
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

int vec_grid(const Ctx* c) { return std::min(c->red_grid, (c->n + kThreads - 1) / kThreads); }

// Grid of the residual update (upd_grid CTAs of kThreads).
int upd_grid(const Ctx* c) { return std::max(1, std::min(c->upd_grid, (c->n / 2 + kThreads - 1) / kThreads)); }

// Grid of the Gram-Schmidt kernels: one CTA per SM, each with several rows
// per thread, so the per-CTA partial sums stay few.
int gs_grid(const Ctx* c) { return std::max(1, std::min(kNumSMs, (c->n + kGsThreads - 1) / kGsThreads)); }

// Dynamic shared memory of the Givens step (column j + 2, rotations 2 j).
size_t gs_stage_bytes(int m) { return sizeof(double) * (3 * size_t(m) + 4); }

// One PCG iteration body (everything after the convergence test is skipped
// once ks->done is set).
gdsw_status pcg_body(Ctx* c, cudaStream_t s, cudaGraphConditionalHandle h, int use_handle) {
  GDSW_TRY(launch_spmv(c, c->p, c->q, s, c->ks));
  k_pcg_update<<<upd_grid(c), kThreads, 0, s>>>(c->n, c->r, c->q, c->red, c->ks, h, use_handle);
  GDSW_CK(cudaGetLastError());
  // x += alpha p is off the path to the next SpMV: it goes on the second
  // stream behind the coarse branch and is joined before p is overwritten
  const bool aside = c->aux_stream != nullptr;
  if (aside) GDSW_CK(cudaEventRecord(c->ev_x, s));
  GDSW_TRY(apply_enqueue(c, c->r, c->z, s, true));
  cudaStream_t xs = aside ? c->aux_stream : s;
  if (aside) GDSW_CK(cudaStreamWaitEvent(xs, c->ev_x, 0));
  k_pcg_xupdate<<<vec_grid(c), kThreads, 0, xs>>>(c->n, c->x, c->p, c->ks);
  GDSW_CK(cudaGetLastError());
  if (aside) {
    GDSW_CK(cudaEventRecord(c->ev_xdone, xs));
    GDSW_CK(cudaStreamWaitEvent(s, c->ev_xdone, 0));
  }
  k_pupdate<<<vec_grid(c), kThreads, 0, s>>>(c->n, c->z, c->p, c->ks);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

gdsw_status read_scalars(Ctx* c, cudaStream_t s) {
  GDSW_CK(cudaMemcpyAsync(c->ks_host, c->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  return GDSW_OK;
}

gdsw_status set_done(Ctx* c, cudaStream_t s, int v) {
  GDSW_CK(cudaMemcpyAsync(&c->ks->done, &v, sizeof(int), cudaMemcpyHostToDevice, s));
  return GDSW_OK;
}

}  // namespace

// Tile height for the stream SpMV: the largest R in {256, 128, 64, 32} whose
// worst tile keeps its products within 64 KB of shared memory; the grid is the
// number of CTAs that fit on the SMs at once.
gdsw_status spmv_configure(Ctx* c, const int* rowptr, const int* colind, const double* val) {
  const int n = c->n;
  // long rows: the sliced ELL copy, beside the CSR kernel (the choice is timed)
  {
    std::vector<int64_t> sptr;
    if (plan_sell(n, rowptr, colind, &sptr)) {
      const int64_t total = sptr.back();
      std::vector<int16_t> scol(static_cast<size_t>(total), 0);
      std::vector<double> sval(static_cast<size_t>(total), 0.0);
      for (int i = 0; i < n; ++i) {
        const int q = i / kSellRows, r = i % kSellRows;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
          const int64_t at = sptr[q] + int64_t(e - rowptr[i]) * kSellRows + r;
          scol[at] = static_cast<int16_t>(colind[e] - i);
          sval[at] = val[e];
        }
      }
      GDSW_TRY(upload(c, &c->sell_ptr, sptr, nullptr));
      GDSW_TRY(upload(c, &c->sell_col, scol, nullptr));
      GDSW_TRY(upload(c, &c->sell_val, sval, nullptr));
      c->sell_slices = static_cast<int>(sptr.size()) - 1;
    }
  }
  // columns as 16-bit offsets from the row when every one fits (the
  // thread-per-row kernel then reads 10 bytes per entry instead of 12)
  {
    bool fits = n > 0;
    for (int i = 0; i < n && fits; ++i)
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colind[e] - i < -32768 || colind[e] - i > 32767) { fits = false; break; }
    if (fits && c->dcol16 == nullptr) {
      std::vector<int16_t> d(static_cast<size_t>(rowptr[n]));
      for (int i = 0; i < n; ++i)
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) d[e] = static_cast<int16_t>(colind[e] - i);
      GDSW_TRY(upload(c, &c->dcol16, d, nullptr));
    }
  }
  // long rows (more than 16 entries on average): W lanes per row, W the power
  // of two nearest to a tenth of the mean row length, within 4..32
  const double mean = n > 0 ? double(rowptr[n]) / n : 0.0;
  c->spmv_W = 0;
  if (mean > 16.0) {
    int W = 4;
    while (W < 32 && W * 10 < mean) W *= 2;
    c->spmv_W = W;
    int per_sm = 1;
    switch (W) {
      case 4: GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv_rows<4>, 256, 0)); break;
      case 8: GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv_rows<8>, 256, 0)); break;
      case 16: GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv_rows<16>, 256, 0)); break;
      default: GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv_rows<32>, 256, 0)); break;
    }
    c->spmv_grid = std::max(1, per_sm) * kNumSMs;
    c->spmv_tiles = 1;
    return GDSW_OK;
  }
  // the thread-per-row kernel keeps the first U entries of a row in flight;
  // U is the longest row (4..8), so no FP64 FMA is issued for an empty slot
  int longest = 0;
  for (int i = 0; i < n; ++i) longest = std::max(longest, rowptr[i + 1] - rowptr[i]);
  c->spmv_U = std::min(8, std::max(4, longest));
  int R = 256, maxne = 0;
  for (; R >= 32; R >>= 1) {
    maxne = 0;
    for (int r0 = 0; r0 < n; r0 += R) maxne = std::max(maxne, rowptr[std::min(n, r0 + R)] - rowptr[r0]);
    if (size_t(maxne) * 2 * sizeof(double) <= 64 * 1024 || R == 32) break;
  }
  if (size_t(maxne) * 2 * sizeof(double) > 200 * 1024) {
    set_error("rows too long for the SpMV tile (%d entries in 32 rows)", maxne);
    return GDSW_ERR_UNSUPPORTED;
  }
  c->spmv_R = R;
  c->spmv_maxne = std::max(1, maxne);
  c->spmv_tiles = (n + R - 1) / R;
  const size_t shm = size_t(c->spmv_maxne) * 2 * sizeof(double);
  int per_sm = 1;
  switch (R) {
#define GDSW_SPMV_CFG(RR)                                                                         \
  case RR:                                                                                         \
    GDSW_CK(allow_max_dynamic_smem(k_spmv_stream<RR>));                                 \
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv_stream<RR>, RR, shm));  \
    break;
    GDSW_SPMV_CFG(256)
    GDSW_SPMV_CFG(128)
    GDSW_SPMV_CFG(64)
    GDSW_SPMV_CFG(32)
#undef GDSW_SPMV_CFG
  }
  c->spmv_grid = std::max(1, per_sm) * kNumSMs;
  return GDSW_OK;
}

namespace {

// Resident CTAs of the tiled SpMV kernels for tile height R: the plain one and
// the one with the next tile's loads in flight.
template <int RR>
gdsw_status spmv_grids(size_t shm, int* g_stream, int* g_pipe) {
  int a = 1, b = 1;
  GDSW_CK(allow_max_dynamic_smem(k_spmv_stream<RR>));
  GDSW_CK(allow_max_dynamic_smem(k_spmv_pipe<RR>));
  GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_spmv_stream<RR>, RR, shm));
  GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmv_pipe<RR>, RR, shm));
  *g_stream = std::max(1, a) * kNumSMs;
  *g_pipe = std::max(1, b) * kNumSMs;
  return GDSW_OK;
}

// Measured choice among the SpMV kernels for short rows (the two tiled ones
// and the one with a thread per row; three timed launches each after a
// warm-up, CUDA events, on the Krylov workspace): all compute the same sums in
// the same order, so the choice changes the speed only.
// GDSW_SPMV=stream|pipe|thread fixes it instead (for profilers).
// The sliced ELL kernel (4 or 8 entries of a lane in flight) against the CSR
// kernel for long rows, three launches each (CUDA events, after one warm-up);
// GDSW_SPMV=sell or sell8 forces the first, any other value the second.
gdsw_status spmv_tune_long(Ctx* c, cudaStream_t s) {
  c->spmv_sell = 0;
  if (c->sell_ptr == nullptr) return GDSW_OK;
  const char* env = getenv("GDSW_SPMV");
  if (env != nullptr) {                 // forced: the sliced ELL kernel only for "sell" / "sell8"
    c->spmv_sell = std::string(env) == "sell" ? 1 : std::string(env) == "sell8" ? 2 : 0;
    return GDSW_OK;
  }
  cudaEvent_t e0, e1;
  GDSW_CK(cudaEventCreate(&e0));
  GDSW_CK(cudaEventCreate(&e1));
  float t[3] = {0.f, 0.f, 0.f};
  gdsw_status st = GDSW_OK;
  for (int k = 0; k < 3 && st == GDSW_OK; ++k) {
    c->spmv_sell = k;
    st = launch_spmv(c, c->p, c->q, s, nullptr);
    if (st != GDSW_OK) break;
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep) st = launch_spmv(c, c->p, c->q, s, nullptr);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], e0, e1);
    if (e != cudaSuccess) { set_error("SpMV tuning: %s", cudaGetErrorString(e)); st = GDSW_ERR_CUDA; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = 0;
  for (int k = 1; k < 3; ++k)
    if (t[k] < t[best]) best = k;
  c->spmv_sell = st == GDSW_OK ? best : 0;
  return st;
}

gdsw_status spmv_tune(Ctx* c, cudaStream_t s) {
  if (c->spmv_W > 0) return spmv_tune_long(c, s);
  const size_t shm = size_t(c->spmv_maxne) * 2 * sizeof(double);
  int g[3] = {c->spmv_grid, c->spmv_grid, c->spmv_grid};
  switch (c->spmv_R) {
    case 256: GDSW_TRY(spmv_grids<256>(shm, &g[0], &g[1])); break;
    case 128: GDSW_TRY(spmv_grids<128>(shm, &g[0], &g[1])); break;
    case 64: GDSW_TRY(spmv_grids<64>(shm, &g[0], &g[1])); break;
    default: GDSW_TRY(spmv_grids<32>(shm, &g[0], &g[1])); break;
  }
  {
    int per_sm = 1;
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv_thread<8, int>, 256, 0));
    g[2] = std::max(1, per_sm) * kNumSMs;
  }
  // the pipelined kernel holds eight entries per thread of a tile
  const bool pipe_ok = c->spmv_maxne <= 8 * c->spmv_R;
  const char* env = getenv("GDSW_SPMV");
  if (env != nullptr) {
    const std::string k(env);
    c->spmv_pipe = (k == "pipe" && pipe_ok) ? 1 : k == "thread" ? 2 : 0;
    c->spmv_grid = g[c->spmv_pipe];
    return GDSW_OK;
  }
  cudaEvent_t e0, e1;
  GDSW_CK(cudaEventCreate(&e0));
  GDSW_CK(cudaEventCreate(&e1));
  float best = 3.4e38f;
  int best_k = 0;
  gdsw_status st = GDSW_OK;
  for (int k = 0; k < 3 && st == GDSW_OK; ++k) {
    if (k == 1 && !pipe_ok) continue;
    c->spmv_pipe = k;
    c->spmv_grid = g[k];
    st = launch_spmv(c, c->p, c->q, s, nullptr);
    if (st != GDSW_OK) break;
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep) st = launch_spmv(c, c->p, c->q, s, nullptr);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { set_error("SpMV tuning: %s", cudaGetErrorString(e)); st = GDSW_ERR_CUDA; break; }
    if (ms < best) { best = ms; best_k = k; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->spmv_pipe = best_k;
  c->spmv_grid = g[best_k];
  return st;
}

}  // namespace

gdsw_status spmv_enqueue(Ctx* c, const double* x, double* y, cudaStream_t s) {
  return launch_spmv(c, x, y, s, nullptr);
}

gdsw_status spmv_enqueue_batch(Ctx* c, const double* x, double* y, cudaStream_t s) {
  return launch_spmv(c, x, y, s, nullptr, batch_gate(c));
}

gdsw_status gmres_cycle(Ctx* c, cudaStream_t s);
gdsw_status gmres_cycle_dc(Ctx* c, cudaStream_t s);

gdsw_status krylov_init(Ctx* c, cudaStream_t s) {
  const int n = c->n;
  c->red_grid = kNumSMs * 8;
  // two CTAs per SM: few partial sums for the last CTA (and few arrivals on
  // its ticket), each thread several trips of kUpdPairs pairs
  c->upd_grid = 2 * kNumSMs;
  if (const char* e = getenv("GDSW_UPD_CTAS_PER_SM")) c->upd_grid = std::max(1, std::min(8, atoi(e))) * kNumSMs;
  // (any SpMV grid: at most 32 resident CTAs per SM)
  c->red_len = std::max(std::max(2 * c->red_grid, 2 * c->nblk), std::max(c->spmv_grid, 32 * kNumSMs)) + 64;
  if (c->opt.krylov == GDSW_KRYLOV_GMRES)
    c->red_len = std::max<int>(c->red_len, (2 * c->opt.restart + 4) * c->red_grid + 64);
  GDSW_TRY(dalloc(c, &c->red, c->red_len));
  GDSW_TRY(dalloc(c, &c->x, n));
  GDSW_TRY(dalloc(c, &c->r, n));
  GDSW_TRY(dalloc(c, &c->z, n));
  GDSW_TRY(dalloc(c, &c->p, n));
  GDSW_TRY(dalloc(c, &c->q, n));
  GDSW_TRY(dalloc(c, &c->b, n));
  GDSW_CK(cudaMemsetAsync(c->z, 0, sizeof(double) * n, s));
  GDSW_CK(cudaMemsetAsync(c->p, 0, sizeof(double) * n, s));
  GDSW_TRY(dalloc(c, &c->ks, 1));
  GDSW_CK(cudaMemsetAsync(c->ks, 0, sizeof(KrylovScalars), s));
  GDSW_CK(cudaMallocHost(&c->ks_host, sizeof(KrylovScalars)));
  if (c->opt.krylov == GDSW_KRYLOV_GMRES) {
    const int m = std::max(1, c->opt.restart);
    GDSW_TRY(dalloc(c, &c->V, size_t(m + 1) * n));
    GDSW_TRY(dalloc(c, &c->Zk, size_t(m) * n));
    GDSW_TRY(dalloc(c, &c->hcol, m + 2));
    GDSW_TRY(dalloc(c, &c->gm, GmLayout(m).total()));
  }
  if (c->opt.krylov == GDSW_KRYLOV_GMRES) {
    // the Givens step's staging in shared memory (more than the default 48 KB
    // only for restarts beyond 2000)
    const size_t gsm = gs_stage_bytes(std::max(1, c->opt.restart));
    if (gsm > size_t(max_block_smem_optin())) {
      set_error("GMRES restart %d too long for the Givens staging", c->opt.restart);
      return GDSW_ERR_UNSUPPORTED;
    }
    if (gsm > 48 * 1024) {
      GDSW_CK(cudaFuncSetAttribute(k_gs_orth1, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(gsm)));
      GDSW_CK(cudaFuncSetAttribute(k_gs_orth2, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(gsm)));
    }
  }
  for (int q = 0; q < 8; ++q) GDSW_CK(cudaEventCreate(&c->ev[q]));
  GDSW_CK(cudaStreamSynchronize(s));
  // the SpMV kernel is chosen by timing before the graphs capture it
  GDSW_TRY(spmv_tune(c, s));
  GDSW_CK(cudaStreamSynchronize(s));
  // the PCG iteration as a graph: while (cond) { body }, cond cleared on device
  const char* env = getenv("GDSW_PCG_GRAPH");
  const bool use_graph = env == nullptr || env[0] != '0';
  if (c->opt.krylov == GDSW_KRYLOV_PCG && use_graph && c->nprob == 1) {
    GDSW_CK(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    GDSW_CK(cudaGraphCreate(&c->pcg_graph, 0));
    cudaGraphConditionalHandle h;
    GDSW_CK(cudaGraphConditionalHandleCreate(&h, c->pcg_graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    GDSW_CK(cudaGraphAddNode(&node, c->pcg_graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    GDSW_CK(cudaStreamBeginCaptureToGraph(c->graph_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    gdsw_status st = pcg_body(c, c->graph_stream, h, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->graph_stream, &captured);
    if (st != GDSW_OK) return st;
    GDSW_CK(e);
    GDSW_CK(cudaGraphInstantiate(&c->pcg_exec, c->pcg_graph, 0));
  }
  // one GMRES restart cycle as a graph (the kernels are gated on the stop flag)
  if (c->opt.krylov == GDSW_KRYLOV_GMRES && use_graph && c->nprob == 1) {
    if (c->graph_stream == nullptr) GDSW_CK(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    GDSW_CK(cudaStreamBeginCapture(c->graph_stream, cudaStreamCaptureModeThreadLocal));
    gdsw_status st = c->opt.gmres_orth == GDSW_GMRES_ORTH_DCGS2 ? gmres_cycle_dc(c, c->graph_stream)
                                                               : gmres_cycle(c, c->graph_stream);
    cudaError_t e = cudaStreamEndCapture(c->graph_stream, &c->gm_graph);
    if (st != GDSW_OK) return st;
    GDSW_CK(e);
    GDSW_CK(cudaGraphInstantiate(&c->gm_exec, c->gm_graph, 0));
  }
  GDSW_TRY(persistent_configure(c));
  return GDSW_OK;
}

gdsw_status solve_pcg(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s) {
  const double t0 = now_s();
  const int n = c->n;
  GDSW_CK(cudaMemcpyAsync(c->b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->x, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  KrylovScalars init = {};
  init.maxit = c->opt.maxit;
  init.flexible = c->flexible ? 1 : 0;
  init.rz = 1.0;
  GDSW_CK(cudaMemcpyAsync(c->ks, &init, sizeof(KrylovScalars), cudaMemcpyHostToDevice, s));
  // r = b - A x0
  GDSW_TRY(launch_spmv(c, c->x, c->q, s, nullptr));
  k_residual<<<vec_grid(c), kThreads, 0, s>>>(n, c->b, c->q, c->r, c->red, c->ks);
  GDSW_CK(cudaGetLastError());
  GDSW_TRY(read_scalars(c, s));
  const double bb = c->ks_host->bb;
  const double tol2 = c->opt.tol * c->opt.tol * bb;
  int iters = 0;
  bool converged = false;
  double rr = c->ks_host->rr;
  if (bb == 0.0) {
    GDSW_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    GDSW_CK(cudaMemsetAsync(c->x, 0, sizeof(double) * n, s));
    GDSW_CK(cudaStreamSynchronize(s));
    if (info) { info->iters = 0; info->converged = 1; info->true_relres = 0.0; info->seconds = now_s() - t0; }
    return GDSW_OK;
  }
  if (rr <= tol2) {
    converged = true;
  } else {
    GDSW_CK(cudaMemcpyAsync(&c->ks->tol2, &tol2, sizeof(double), cudaMemcpyHostToDevice, s));
    // z = M r, (r, z), p = z
    GDSW_TRY(apply_enqueue(c, c->r, c->z, s, true));
    GDSW_CK(cudaMemcpyAsync(c->p, c->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    for (;;) {
      if (c->persist_grid > 0) {
        GDSW_TRY(pcg_persistent_run(c, s));
        // a grid barrier that ran out ends the solve (GDSW_ERR_TIMEOUT)
        GDSW_TRY(check_device_errors(c, s));
      } else if (c->pcg_exec != nullptr) {
        GDSW_CK(cudaGraphLaunch(c->pcg_exec, s));
      } else {
        // the same iteration body launched from the host (no CUDA graph), with
        // the stop flag read back after every iteration
        for (;;) {
          GDSW_TRY(pcg_body(c, s, cudaGraphConditionalHandle{}, 0));
          GDSW_TRY(read_scalars(c, s));
          if (c->ks_host->done) break;
        }
      }
      // recompute the true residual where the recurrence says converged (or maxit)
      GDSW_TRY(launch_spmv(c, c->x, c->q, s, nullptr));
      k_residual<<<vec_grid(c), kThreads, 0, s>>>(n, c->b, c->q, c->r, c->red, c->ks);
      GDSW_CK(cudaGetLastError());
      GDSW_TRY(read_scalars(c, s));
      iters = c->ks_host->iter;
      rr = c->ks_host->rr;
      if (rr <= tol2) { converged = true; break; }
      if (c->ks_host->bad || iters >= c->opt.maxit || !std::isfinite(rr)) break;
      // continue from the true residual: z = M r, beta, p = z + beta p
      GDSW_TRY(set_done(c, s, 0));
      GDSW_TRY(apply_enqueue(c, c->r, c->z, s, true));
      k_pupdate<<<vec_grid(c), kThreads, 0, s>>>(n, c->z, c->p, c->ks);
      GDSW_CK(cudaGetLastError());
    }
  }
  GDSW_CK(cudaMemcpyAsync(x, c->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaStreamSynchronize(s));
  GDSW_TRY(check_device_errors(c, s));
  if (info) {
    info->iters = iters;
    info->converged = converged ? 1 : 0;
    info->true_relres = std::sqrt(rr / bb);
    info->seconds = now_s() - t0;
  }
  if (!converged) { set_error("PCG stopped after %d iterations at relative residual %.3e", iters, std::sqrt(rr / bb)); return GDSW_ERR_NOT_CONVERGED; }
  return GDSW_OK;
}

gdsw_status pcg_iteration_timed(Ctx* c, const double* b, cudaStream_t s, double* ms) {
  if (c->nprob != 1) { set_error("timed PCG iteration: batched handles are not supported"); return GDSW_ERR_UNSUPPORTED; }
  const int n = c->n;
  KrylovScalars init = {};
  init.maxit = 1 << 30;
  init.flexible = c->flexible ? 1 : 0;
  init.rz = 1.0;
  init.tol2 = -1.0;                          // never met: the timed iteration runs every kernel
  GDSW_CK(cudaMemcpyAsync(c->ks, &init, sizeof(KrylovScalars), cudaMemcpyHostToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemsetAsync(c->x, 0, sizeof(double) * n, s));
  GDSW_CK(cudaMemcpyAsync(c->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_TRY(apply_enqueue(c, c->r, c->z, s, true));
  GDSW_CK(cudaMemcpyAsync(c->p, c->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  cudaEvent_t ev[9] = {};
  gdsw_status st = GDSW_OK;
  for (int q = 0; q < 9 && st == GDSW_OK; ++q)
    if (cudaEventCreate(&ev[q]) != cudaSuccess) { set_error("event creation failed"); st = GDSW_ERR_CUDA; }
  cudaEvent_t* ap = ev + 2;                  // the apply records ap[0..4]
  if (st == GDSW_OK) {
    cudaEventRecord(ev[0], s);
    st = launch_spmv(c, c->p, c->q, s, c->ks);
  }
  if (st == GDSW_OK) {
    cudaEventRecord(ev[1], s);
    k_pcg_update<<<upd_grid(c), kThreads, 0, s>>>(n, c->r, c->q, c->red, c->ks, cudaGraphConditionalHandle{}, 0);
    if (cudaGetLastError() != cudaSuccess) { set_error("vector update launch failed"); st = GDSW_ERR_CUDA; }
  }
  if (st == GDSW_OK) st = apply_timed_dots(c, c->r, c->z, s, ap);
  if (st == GDSW_OK) {
    // one stream: the x update after the apply, then p
    k_pcg_xupdate<<<vec_grid(c), kThreads, 0, s>>>(n, c->x, c->p, c->ks);
    cudaEventRecord(ev[7], s);
    k_pupdate<<<vec_grid(c), kThreads, 0, s>>>(n, c->z, c->p, c->ks);
    cudaEventRecord(ev[8], s);
    if (cudaEventSynchronize(ev[8]) != cudaSuccess) { set_error("timed iteration failed"); st = GDSW_ERR_CUDA; }
  }
  if (st == GDSW_OK) st = check_device_errors(c, s);
  if (st == GDSW_OK) {
    // spmv, update, local, phiT, coarse, combine (events ev[0..6]), pupdate, x update
    const int from[8] = {0, 1, 2, 3, 4, 5, 7, 6}, to[8] = {1, 2, 3, 4, 5, 6, 8, 7};
    for (int q = 0; q < 8; ++q) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[from[q]], ev[to[q]]);
      ms[q] = t;
    }
  }
  for (int q = 0; q < 9; ++q)
    if (ev[q]) cudaEventDestroy(ev[q]);
  return st;
}

// One restart cycle of GMRES(m): m Arnoldi steps, each z_j = M^-1 v_j,
// w = A z_j, one fused reduction for V^T w and (w, w), the orthogonalisation
// (a second pass only when the first cancelled), and the Givens update; every
// kernel is gated on the stop flag, so the cycle can be enqueued (or captured)
// whole and ends early on convergence without a host round trip.
gdsw_status gmres_cycle(Ctx* c, cudaStream_t s) {
  const int n = c->n;
  // two passes always (CGS2), or one pass with a second only where the
  // Pythagorean norm cancels (single reduction per step)
  c->gm_keep = c->opt.gmres_orth == GDSW_GMRES_ORTH_SINGLE ? 1e-4 : 2.0;
  const int m = std::max(1, c->opt.restart);
  const GmLayout L(m);
  double* h1 = c->gm + L.h1();
  double* h2 = c->gm + L.h2();
  double* bt = c->gm + L.beta();
  const int Ggs = gs_grid(c);
  const size_t gsm = gs_stage_bytes(m);
  for (int j = 0; j < m; ++j) {
    const int k = j + 1;
    double* vj = c->V + int64_t(j) * n;
    double* zj = c->Zk + int64_t(j) * n;
    double* w = c->V + int64_t(k) * n;
    GDSW_TRY(apply_enqueue_gated(c, vj, zj, s));
    GDSW_TRY(launch_spmv(c, zj, w, s, c->ks));
    k_gs_pass1<<<Ggs, kGsThreads, 0, s>>>(n, k, c->V, w, c->red, h1, bt, c->ks, c->gm_keep);
    k_gs_orth1<<<Ggs, kGsThreads, gsm, s>>>(n, k, c->V, h1, bt, w, c->red, h2, j, m, c->gm, c->ks);
    k_gs_orth2<<<Ggs, kGsThreads, gsm, s>>>(n, k, c->V, h2, bt, w, j, m, c->gm, c->ks);
    GDSW_CK(cudaGetLastError());
  }
  return GDSW_OK;
}

// One restart cycle with delayed reorthogonalisation: per step the apply, the
// SpMV, one launch for the fused reduction and the scalar step (k_dc_step),
// and one vector pass; a last reduction finishes the final column.  u, M^-1 u and w live in the PCG
// vectors p, z and q; the driver has put q_0 = r / beta in V_0.
gdsw_status gmres_cycle_dc(Ctx* c, cudaStream_t s) {
  const int n = c->n;
  const int m = std::max(1, c->opt.restart);
  const int Ggs = gs_grid(c);
  double* u = c->p;
  double* zu = c->z;
  double* w = c->q;
  GDSW_CK(cudaMemcpyAsync(u, c->V, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < m; ++k) {
    GDSW_TRY(apply_enqueue_gated(c, u, zu, s));
    GDSW_TRY(launch_spmv(c, zu, w, s, c->ks));
    k_dc_step<<<Ggs, kGsThreads, 0, s>>>(n, k, m, c->V, u, w, c->red, c->gm, c->ks, 0);
    k_dc_update<<<Ggs, kGsThreads, 0, s>>>(n, k, m, c->V, c->Zk, u, zu, w, c->gm, c->ks);
    GDSW_CK(cudaGetLastError());
  }
  k_dc_step<<<Ggs, kGsThreads, 0, s>>>(n, m, m, c->V, u, nullptr, c->red, c->gm, c->ks, 1);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

// Right-preconditioned restarted GMRES(m) (Sec. VII) with the Arnoldi
// process, the Hessenberg matrix and the Givens rotations on the device: each
// Gram-Schmidt pass is one fused reduction (V^T w together with (w, w)); two
// passes (CGS2) by default, or the single-reduce form (one pass, a second
// only on cancellation).  One host round trip per restart cycle, where the
// true residual is recomputed and the small triangular system is solved.
gdsw_status solve_gmres(Ctx* c, const double* b, double* x, gdsw_solve_info* info, cudaStream_t s) {
  const double t0 = now_s();
  const int n = c->n;
  const int m = std::max(1, c->opt.restart);
  const int G = vec_grid(c);
  const GmLayout L(m);
  GDSW_CK(cudaMemcpyAsync(c->b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaMemcpyAsync(c->x, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  KrylovScalars init = {};
  init.maxit = c->opt.maxit;
  GDSW_CK(cudaMemcpyAsync(c->ks, &init, sizeof(KrylovScalars), cudaMemcpyHostToDevice, s));
  std::vector<double> gmh(L.total());
  int it = 0;
  double bb = 0.0, rr = 0.0;
  bool converged = false;
  for (;;) {
    GDSW_TRY(launch_spmv(c, c->x, c->q, s, nullptr));
    k_residual<<<G, kThreads, 0, s>>>(n, c->b, c->q, c->r, c->red, c->ks);
    GDSW_CK(cudaGetLastError());
    GDSW_TRY(read_scalars(c, s));
    bb = c->ks_host->bb;
    rr = c->ks_host->rr;
    if (bb == 0.0) {
      GDSW_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
      GDSW_CK(cudaMemsetAsync(c->x, 0, sizeof(double) * n, s));
      GDSW_CK(cudaStreamSynchronize(s));
      if (info) { info->iters = 0; info->converged = 1; info->true_relres = 0; info->seconds = now_s() - t0; }
      return GDSW_OK;
    }
    const double tolabs = c->opt.tol * std::sqrt(bb);
    const double beta = std::sqrt(rr);
    if (beta <= tolabs) { converged = true; break; }
    if (it >= c->opt.maxit || !std::isfinite(beta) || c->ks_host->bad) break;
    // V_0 = r / beta; g = (beta, 0, ...); the cycle's stop flag cleared
    const double inv = 1.0 / beta;
    GDSW_CK(cudaMemcpyAsync(c->hcol, &inv, sizeof(double), cudaMemcpyHostToDevice, s));
    k_scale_copy<<<G, kThreads, 0, s>>>(n, c->r, c->hcol, c->V);
    std::fill(gmh.begin(), gmh.end(), 0.0);
    gmh[L.g()] = beta;
    GDSW_CK(cudaMemcpyAsync(c->gm, gmh.data(), sizeof(double) * L.total(), cudaMemcpyHostToDevice, s));
    KrylovScalars* kh = c->ks_host;
    kh->done = 0;
    kh->iter = it;
    kh->tol2 = tolabs * tolabs;
    kh->gm_mode = 1;
    GDSW_CK(cudaMemcpyAsync(c->ks, kh, sizeof(KrylovScalars), cudaMemcpyHostToDevice, s));
    if (c->gm_exec != nullptr) GDSW_CK(cudaGraphLaunch(c->gm_exec, s));
    else if (c->opt.gmres_orth == GDSW_GMRES_ORTH_DCGS2) GDSW_TRY(gmres_cycle_dc(c, s));
    else GDSW_TRY(gmres_cycle(c, s));
    GDSW_CK(cudaMemcpyAsync(gmh.data(), c->gm, sizeof(double) * L.total(), cudaMemcpyDeviceToHost, s));
    GDSW_TRY(read_scalars(c, s));
    const int jdone = c->ks_host->iter - it;
    it = c->ks_host->iter;
    if (jdone > 0) {
      // y = R^-1 g, x += Z y
      std::vector<double> yv(jdone);
      for (int i = jdone - 1; i >= 0; --i) {
        double v = gmh[L.g() + i];
        for (int k = i + 1; k < jdone; ++k) v -= gmh[size_t(i) * m + k] * yv[k];
        yv[i] = v / gmh[size_t(i) * m + i];
      }
      GDSW_CK(cudaMemcpyAsync(c->hcol, yv.data(), sizeof(double) * jdone, cudaMemcpyHostToDevice, s));
      k_update_x<<<G, kThreads, 0, s>>>(n, jdone, c->Zk, c->hcol, c->x);
      GDSW_CK(cudaGetLastError());
    }
    if (c->ks_host->bad || jdone == 0) {
      // breakdown without progress: recompute the residual once more and stop
      GDSW_TRY(launch_spmv(c, c->x, c->q, s, nullptr));
      k_residual<<<G, kThreads, 0, s>>>(n, c->b, c->q, c->r, c->red, c->ks);
      GDSW_CK(cudaGetLastError());
      GDSW_TRY(read_scalars(c, s));
      rr = c->ks_host->rr;
      converged = std::sqrt(rr) <= tolabs;
      break;
    }
  }
  GDSW_CK(cudaMemcpyAsync(x, c->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GDSW_CK(cudaStreamSynchronize(s));
  GDSW_TRY(check_device_errors(c, s));
  if (info) {
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->true_relres = std::sqrt(rr / bb);
    info->seconds = now_s() - t0;
  }
  if (!converged) { set_error("GMRES stopped after %d iterations", it); return GDSW_ERR_NOT_CONVERGED; }
  return GDSW_OK;
}

}  // namespace gdsw
