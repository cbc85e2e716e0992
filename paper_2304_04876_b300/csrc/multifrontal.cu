// Multifrontal exact local solver on the device (Sec. V-B1 exact local
// solves; the triangular sweeps by the partitioned inverse of Sec. V-B2).
//
// Factorisation (setup, FP64): one CTA per subdomain walks its supernodes in
// postorder.  Each front S u B(S) is assembled from A_s and the children's
// update matrices, the first |S| columns are factored (right-looking, the
// pivot column staged in shared memory), the Schur complement goes to the
// subdomain's update stack for the parent, and L_SS is inverted.  The panel
// [Linv_SS; L_BS] is stored in the apply precision.
//
// Solve (every apply): one CTA per subdomain, the local vector in shared
// memory in nested-dissection order, the tree walked one level (height) at a
// time.  Forward:  f_S += children's update vectors;  y_S = Linv_SS f_S;
// u_S = (children's contributions on B(S)) - L_BS y_S.  Backward (top down):
// g_S = y_S - L_BS^T x_B;  x_S = Linv_SS^T g_S.  Every step is a dense
// matrix-vector product on a column-major panel, coalesced in both
// directions (rows in the forward sweep, column dot products in the backward
// one), and every sum runs in a fixed order.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <type_traits>

#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace gdsw {

namespace {

enum { MF_ERR_BREAKDOWN = 1 };

template <class T>
__device__ __forceinline__ T to_storage(double x) { return T(x); }
template <>
__device__ __forceinline__ __half to_storage<__half>(double x) { return __double2half(x); }

template <class T>
__device__ __forceinline__ float ld_f(const T* p) { return float(*p); }
__device__ __forceinline__ double ld_f(const double* p) { return *p; }
template <>
__device__ __forceinline__ float ld_f<__half>(const __half* p) { return __half2float(*p); }

__device__ __forceinline__ int64_t mf_col(int nf, int j) {
  return int64_t(j) * nf - int64_t(j) * (j - 1) / 2;
}

// ---------------------------------------------------------------------------
// factorisation
// ---------------------------------------------------------------------------
struct MfFactorArgs {
  const MfSn* sn;
  const int* sub_sn;
  const int* ch_ptr;
  const int* ch_list;
  const uint16_t* relF;
  const int* asm_ptr;
  const int* asm_ent;
  const uint32_t* asm_rc;
  const int64_t* stack_off;
  const double* araw;       // values of every A_s entry
  double* work;             // per CTA: front, inverse block, update stack
  const int64_t* work_off;  // per CTA of the batch
  int64_t front_len;        // max front^2
  int64_t inv_len;          // max |S|^2
  int q0;
  int* err;
};

template <class T>
__global__ void __launch_bounds__(512) k_mf_factor(MfFactorArgs a, T* __restrict__ panel) {
  extern __shared__ double colv[];   // pivot column of the front being factored
  __shared__ double piv_sh;
  const int q = a.q0 + blockIdx.x;
  double* F = a.work + a.work_off[blockIdx.x];
  double* X = F + a.front_len;
  double* stack = X + a.inv_len;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int S = a.sub_sn[q]; S < a.sub_sn[q + 1]; ++S) {
    const MfSn d = a.sn[S];
    const int ns = d.ns, nb = d.nb, nf = ns + nb;
    for (int64_t t = threadIdx.x; t < int64_t(nf) * nf; t += blockDim.x) F[t] = 0.0;
    __syncthreads();
    for (int e = a.asm_ptr[S] + threadIdx.x; e < a.asm_ptr[S + 1]; e += blockDim.x) {
      const uint32_t rc = a.asm_rc[e];
      F[int64_t(rc >> 16) * nf + (rc & 0xffffu)] = a.araw[a.asm_ent[e]];
    }
    __syncthreads();
    // extend-add, one child at a time (a fixed order of the sums)
    for (int t = a.ch_ptr[S]; t < a.ch_ptr[S + 1]; ++t) {
      const MfSn dc = a.sn[a.ch_list[t]];
      const double* U = stack + a.stack_off[a.ch_list[t]];
      const uint16_t* rel = a.relF + dc.brow;
      for (int k = wid; k < dc.nb; k += nw) {
        const int64_t fk = int64_t(rel[k]) * nf;
        for (int r = k + lane; r < dc.nb; r += 32) F[fk + rel[r]] += U[int64_t(k) * dc.nb + r];
      }
      __syncthreads();
    }
    // partial Cholesky of the first ns columns; the trailing update also
    // forms the Schur complement F_BB - L_BS L_BS^T
    for (int j = 0; j < ns; ++j) {
      double* Fj = F + int64_t(j) * nf;
      if (threadIdx.x == 0) {
        const double p = Fj[j];
        if (!(p > 0.0)) { atomicOr(a.err, MF_ERR_BREAKDOWN); piv_sh = 1.0; }
        else piv_sh = sqrt(p);
        Fj[j] = piv_sh;
      }
      __syncthreads();
      const double piv = piv_sh;
      for (int i = j + 1 + threadIdx.x; i < nf; i += blockDim.x) {
        const double v = Fj[i] / piv;
        Fj[i] = v;
        colv[i] = v;
      }
      __syncthreads();
      for (int k = j + 1 + wid; k < nf; k += nw) {
        double* Fk = F + int64_t(k) * nf;
        const double lk = colv[k];
        for (int i = k + lane; i < nf; i += 32) Fk[i] -= colv[i] * lk;
      }
      __syncthreads();
    }
    // Schur complement to the stack (the children's matrices it overlaps are consumed)
    double* US = stack + a.stack_off[S];
    for (int k = wid; k < nb; k += nw)
      for (int r = k + lane; r < nb; r += 32) US[int64_t(k) * nb + r] = F[int64_t(ns + k) * nf + ns + r];
    // Linv_SS: X = L_SS^-1 by rows, every column of the identity at once
    for (int c = wid; c < ns; c += nw)
      for (int i = c + lane; i < ns; i += 32) X[int64_t(c) * ns + i] = i == c ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < ns; ++k) {
      const double lkk = F[int64_t(k) * nf + k];
      for (int c = threadIdx.x; c <= k; c += blockDim.x) X[int64_t(c) * ns + k] /= lkk;
      __syncthreads();
      const double* Lk = F + int64_t(k) * nf;
      for (int c = wid; c <= k; c += nw) {
        double* Xc = X + int64_t(c) * ns;
        const double xk = Xc[k];
        for (int i = k + 1 + lane; i < ns; i += 32) Xc[i] -= Lk[i] * xk;
      }
      __syncthreads();
    }
    // panel [Linv_SS; L_BS], column-major trapezoid
    T* Pn = panel + d.panel;
    for (int j = wid; j < ns; j += nw) {
      T* col = Pn + mf_col(nf, j) - j;
      for (int i = j + lane; i < ns; i += 32) col[i] = to_storage<T>(X[int64_t(j) * ns + i]);
      for (int r = lane; r < nb; r += 32) col[ns + r] = to_storage<T>(F[int64_t(j) * nf + ns + r]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
struct MfSolveArgs {
  const int* om_ptr;
  const int* sub_lv;
  const int64_t* sub_panel;  // first panel element of each subdomain
  const int* sub_brow;       // first B row of each subdomain
  const MfLevel* lv;
  const uint16_t* rows;
  const uint16_t* brows;
  const uint32_t* st;        // kMfTaskWords per task
  const uint32_t* xt;
  const uint32_t* ut;
  const int* nd_dof;
  const uint16_t* nd_loc;
  const int* pullS_ptr;
  const int* pullB_ptr;
  const uint16_t* pullS;
  const uint16_t* pullB;
  const uint16_t* bidx;
  int arena;                 // entries of one subdomain's update-vector arena
  int vlen;                  // shared-memory entries of the local vector
  int stage;                 // shared-memory entries of the large supernodes' stage
  int* err;
  long long wait_cycles;
};

struct MfTask {
  uint32_t panel, brow;      // relative to the subdomain's first panel element / B row
  int pos0, ns, nb, stage, uoff, c0;
};

struct MfWords {
  uint32_t w[kMfTaskWords];
};

__device__ __forceinline__ MfWords mf_words(const uint32_t* T5, int t) {
  MfWords x;
  const uint32_t* w = T5 + size_t(t) * kMfTaskWords;
#pragma unroll
  for (int k = 0; k < kMfTaskWords; ++k) x.w[k] = __ldg(w + k);
  return x;
}

__device__ __forceinline__ MfTask mf_decode(const MfWords& x) {
  MfTask d;
  d.panel = x.w[0];
  d.brow = x.w[1];
  const uint32_t w2 = x.w[2], w3 = x.w[3], w4 = x.w[4];
  d.pos0 = int(w2 & 0xffffu);
  d.ns = int(w2 >> 16);
  d.nb = int(w3 & 0xffffu);
  d.stage = int(w3 >> 16);
  d.uoff = int(w4 & 0xffffu);
  d.c0 = int(w4 >> 16);
  return d;
}

__device__ __forceinline__ MfTask mf_task(const uint32_t* T5, int t) { return mf_decode(mf_words(T5, t)); }

// Offset of entry (i, j) of a trapezoid panel with nf rows, less i:
// column j starts at j*nf - j(j-1)/2 and holds rows j .. nf-1.
__device__ __forceinline__ int mf_cofs(int nf, int j) { return j * (nf - 1) - (j * (j - 1)) / 2; }

constexpr int kMfUnroll = 8;   // independent panel loads in flight per lane (large supernodes)
constexpr int kMfK = kMfSmallNb / 32;   // B rows per lane of a small supernode

// Stage a small supernode's panel in this warp's buffer (one bulk copy).
template <class T>
__device__ __forceinline__ void mf_fetch(const T* src, int entries, T* buf, uint64_t* bar) {
  if ((threadIdx.x & 31) == 0) {
    const unsigned bytes = unsigned((entries + 7) & ~7) * sizeof(T);
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    bulk_g2s(buf, src, bytes, bar);
  }
}

// Wait for the warp's staged panel.  A wait that runs out is recorded (the
// host reports GDSW_ERR_TIMEOUT), followed by one more bounded wait for the copy
// to land, and returns false: the warp then issues no further copy, so none is
// left in flight when the CTA ends.
__device__ __forceinline__ bool mf_wait(uint64_t* bar, unsigned& phase, const MfSolveArgs& a) {
  bool ok = true;
  if (!mbar_wait_bounded(bar, phase, a.wait_cycles)) {
    if ((threadIdx.x & 31) == 0) atomicOr(a.err, 1);
    mbar_wait_bounded(bar, phase, kDefaultWaitCycles);
    ok = false;
  }
  phase ^= 1u;
  return ok;
}

template <class T, class TS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_local_mf(const double* __restrict__ r, MfSolveArgs a,
                                                     const TS* __restrict__ panel_all, T* __restrict__ arena_all,
                                                     T* __restrict__ zloc, const KrylovScalars* __restrict__ ks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (ks != nullptr && ks->done) return;
  constexpr int kBufBytes = mf_buf_bytes(int(sizeof(T)));   // this warp's panel buffer
  constexpr int kBufT = kBufBytes / int(sizeof(T));         // x_B gathers

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  T* v = reinterpret_cast<T*>(smem_raw + 64 * sizeof(uint64_t));
  T* stage = v + a.vlen;
  TS* buf = reinterpret_cast<TS*>(reinterpret_cast<unsigned char*>(stage + a.stage) + wid * kBufBytes);
  T* bufT = reinterpret_cast<T*>(buf);             // the same buffer for x_B gathers
  uint64_t* bar = bars + wid;
  if (lane == 0) mbar_init(bar, 1);
  fence_mbar_init();
  unsigned phase = 0;
  bool copies_ok = true;                           // false once a copy wait ran out
  const int q = blockIdx.x;
  const int base = a.om_ptr[q], m = a.om_ptr[q + 1] - base;
  const TS* panel = panel_all + a.sub_panel[q];
  const uint16_t* bidx = a.bidx + a.sub_brow[q];
  const int* pullB_ptr = a.pullB_ptr + a.sub_brow[q];
  T* arena = arena_all + int64_t(q) * a.arena;
  for (int p = tid; p < m; p += nt) v[p] = narrow_bits<T>(load_bits(r, a.nd_dof[base + p]));
  __syncthreads();
  const int l0 = a.sub_lv[q], l1 = a.sub_lv[q + 1];
  // ---- forward sweep, leaves first ----
  for (int l = l0; l < l1; ++l) {
    const MfLevel L = a.lv[l], E = a.lv[l + 1];
    if (L.flags & 1) {
      // f_S += the children's update vectors on S
      for (int t = L.rows + tid; t < E.rows; t += nt) {
        const int p = a.rows[t];
        T acc = v[p];
        for (int k = a.pullS_ptr[base + p]; k < a.pullS_ptr[base + p + 1]; ++k) acc += arena[a.pullS[k]];
        v[p] = acc;
      }
      __syncthreads();
    }
    // small supernodes, one warp each: y_S = Linv_SS f_S, u_S = pulls - L_BS y_S
    MfWords nx;
    if (L.st + wid < E.st) nx = mf_words(a.st, L.st + wid);
    for (int t = L.st + wid; t < E.st && copies_ok; t += nw) {
      const MfTask d = mf_decode(nx);
      const int nf = d.ns + d.nb;
      mf_fetch(panel + d.panel, d.ns * nf - d.ns * (d.ns - 1) / 2, buf, bar);
      if (t + nw < E.st) nx = mf_words(a.st, t + nw);     // the next task's layout, early
      const T f = lane < d.ns ? v[d.pos0 + lane] : T(0);
      T u[kMfK];
#pragma unroll
      for (int k = 0; k < kMfK; ++k) {
        const int rr = lane + 32 * k;
        u[k] = T(0);
        if (rr < d.nb)
          for (int e = pullB_ptr[d.brow + rr]; e < pullB_ptr[d.brow + rr + 1]; ++e) u[k] += arena[a.pullB[e]];
      }
      copies_ok = mf_wait(bar, phase, a) && copies_ok;
      T y = T(0);
      int c = 0;                                   // column j starts at buf + c + j
      for (int j = 0; j < d.ns; ++j) {
        const T fj = __shfl_sync(0xffffffffu, f, j);
        if (lane >= j && lane < d.ns) y += T(ld_f(buf + c + lane)) * fj;
        const T yj = __shfl_sync(0xffffffffu, y, j);   // row j is complete after column j
#pragma unroll
        for (int k = 0; k < kMfK; ++k)
          if (lane + 32 * k < d.nb) u[k] -= T(ld_f(buf + c + d.ns + lane + 32 * k)) * yj;
        c += nf - 1 - j;
      }
      if (lane < d.ns) v[d.pos0 + lane] = y;
#pragma unroll
      for (int k = 0; k < kMfK; ++k)
        if (lane + 32 * k < d.nb) arena[d.uoff + lane + 32 * k] = u[k];
      __syncwarp();
    }
    // large supernodes: 32-row pieces of y_S to the stage
    for (int t = L.xt + wid; t < E.xt; t += nw) {
      const MfTask d = mf_task(a.xt, t);
      const int i0 = d.c0, i = i0 + lane;
      const int nf = d.ns + d.nb, jend = min(i0 + 32, d.ns);
      const bool row = i < d.ns;
      const TS* p = panel + d.panel + i;
      const T* f = v + d.pos0;
      T acc = T(0);
      int j = 0;
      for (; j + kMfUnroll <= jend; j += kMfUnroll) {
        T x[kMfUnroll];
#pragma unroll
        for (int k = 0; k < kMfUnroll; ++k) x[k] = (row && j + k <= i) ? T(ld_f(p + mf_cofs(nf, j + k))) : T(0);
#pragma unroll
        for (int k = 0; k < kMfUnroll; ++k) acc += x[k] * f[j + k];
      }
      for (; j < jend; ++j)
        if (row && j <= i) acc += T(ld_f(p + mf_cofs(nf, j))) * f[j];
      if (row) stage[d.stage + i] = acc;
    }
    if (L.flags & 2) {
      __syncthreads();
      // large supernodes: u_S = children's contributions on B(S) - L_BS y_S
      for (int t = L.ut + wid; t < E.ut; t += nw) {
        const MfTask d = mf_task(a.ut, t);
        const int rr = d.c0 + lane;
        const bool row = rr < d.nb;
        const int nf = d.ns + d.nb;
        const int k0 = row ? pullB_ptr[d.brow + rr] : 0, k1 = row ? pullB_ptr[d.brow + rr + 1] : 0;
        const TS* p = panel + d.panel + d.ns + rr;
        const T* y = stage + d.stage;
        T acc = T(0);
        int j = 0;
        for (; j + 2 * kMfUnroll <= d.ns; j += 2 * kMfUnroll) {   // sixteen loads in flight
          T x[2 * kMfUnroll];
#pragma unroll
          for (int k = 0; k < 2 * kMfUnroll; ++k) x[k] = row ? T(ld_f(p + mf_cofs(nf, j + k))) : T(0);
#pragma unroll
          for (int k = 0; k < 2 * kMfUnroll; ++k) acc -= x[k] * y[j + k];
        }
        for (; j < d.ns; ++j)
          if (row) acc -= T(ld_f(p + mf_cofs(nf, j))) * y[j];
        T pulled = T(0);
        for (int k = k0; k < k1; ++k) pulled += arena[a.pullB[k]];
        if (row) arena[d.uoff + rr] = pulled + acc;
      }
      for (int t = L.br + tid; t < E.br; t += nt) v[a.brows[t]] = stage[t - L.br];
    }
    __syncthreads();
  }
  // ---- backward sweep, root first ----
  for (int l = l1 - 1; l >= l0; --l) {
    const MfLevel L = a.lv[l], E = a.lv[l + 1];
    // small supernodes: g_S = y_S - L_BS^T x_B, x_S = Linv_SS^T g_S, one column per lane
    MfWords nx;
    if (L.st + wid < E.st) nx = mf_words(a.st, L.st + wid);
    for (int t = L.st + wid; t < E.st && copies_ok; t += nw) {
      const MfTask d = mf_decode(nx);
      const int nf = d.ns + d.nb;
      mf_fetch(panel + d.panel, d.ns * nf - d.ns * (d.ns - 1) / 2, buf, bar);
      if (t + nw < E.st) nx = mf_words(a.st, t + nw);
      T xv[kMfK];
#pragma unroll
      for (int k = 0; k < kMfK; ++k) {
        const int rr = lane + 32 * k;
        xv[k] = rr < d.nb ? v[bidx[d.brow + rr]] : T(0);
      }
      const bool col = lane < d.ns;
      T g = col ? v[d.pos0 + lane] : T(0);
      const int cl = col ? mf_cofs(nf, lane) : 0;   // this lane's column
      copies_ok = mf_wait(bar, phase, a) && copies_ok;
#pragma unroll
      for (int k = 0; k < kMfK; ++k) {
        if (32 * k >= d.nb) break;
        const int rend = min(32, d.nb - 32 * k);
        const TS* pc = buf + cl + d.ns + 32 * k;
        for (int r2 = 0; r2 < rend; ++r2) {
          const T xr = __shfl_sync(0xffffffffu, xv[k], r2);
          if (col) g -= T(ld_f(pc + r2)) * xr;
        }
      }
      T x = T(0);
      for (int i = 0; i < d.ns; ++i) {
        const T gi = __shfl_sync(0xffffffffu, g, i);
        if (col && lane <= i) x += T(ld_f(buf + cl + i)) * gi;
      }
      if (col) v[d.pos0 + lane] = x;
      __syncwarp();
    }
    // large supernodes: g_S on 32-column pieces, eight columns at a time; x_B
    // is gathered once per piece into the warp's buffer when it fits
    for (int t = L.xt + wid; t < E.xt; t += nw) {
      const MfTask d = mf_task(a.xt, t);
      if (d.nb == 0) continue;
      const int i0 = d.c0, iend = min(i0 + 32, d.ns), nf = d.ns + d.nb;
      const bool staged = d.nb <= kBufT;
      if (staged)
        for (int rr = lane; rr < d.nb; rr += 32) bufT[rr] = v[bidx[d.brow + rr]];
      __syncwarp();
      for (int i = i0; i < iend; i += kMfUnroll) {
        T acc[kMfUnroll];
#pragma unroll
        for (int k = 0; k < kMfUnroll; ++k) acc[k] = T(0);
        const TS* p = panel + d.panel + d.ns;
        int rr = lane;
        for (; rr + 32 < d.nb; rr += 64) {    // two rows per lane in flight
          T x[kMfUnroll], x2[kMfUnroll];
#pragma unroll
          for (int k = 0; k < kMfUnroll; ++k) {
            const bool c = i + k < iend;
            x[k] = c ? T(ld_f(p + mf_cofs(nf, i + k) + rr)) : T(0);
            x2[k] = c ? T(ld_f(p + mf_cofs(nf, i + k) + rr + 32)) : T(0);
          }
          const T xv = staged ? bufT[rr] : v[bidx[d.brow + rr]];
          const T xv2 = staged ? bufT[rr + 32] : v[bidx[d.brow + rr + 32]];
#pragma unroll
          for (int k = 0; k < kMfUnroll; ++k) acc[k] += x[k] * xv + x2[k] * xv2;
        }
        if (rr < d.nb) {
          T x[kMfUnroll];
#pragma unroll
          for (int k = 0; k < kMfUnroll; ++k) x[k] = (i + k < iend) ? T(ld_f(p + mf_cofs(nf, i + k) + rr)) : T(0);
          const T xv = staged ? bufT[rr] : v[bidx[d.brow + rr]];
#pragma unroll
          for (int k = 0; k < kMfUnroll; ++k) acc[k] += x[k] * xv;
        }
#pragma unroll
        for (int k = 0; k < kMfUnroll; ++k) {
          const T sum = warp_sum(acc[k]);
          if (lane == 0 && i + k < iend) v[d.pos0 + i + k] -= sum;
        }
      }
      __syncwarp();
    }
    if (L.flags & 2) {
      __syncthreads();
      // large supernodes: x_S = Linv_SS^T g_S, eight columns at a time
      for (int t = L.xt + wid; t < E.xt; t += nw) {
        const MfTask d = mf_task(a.xt, t);
        const int j0 = d.c0, jend = min(j0 + 32, d.ns), nf = d.ns + d.nb;
        const T* g = v + d.pos0;
        for (int j = j0; j < jend; j += kMfUnroll) {
          T acc[kMfUnroll];
#pragma unroll
          for (int k = 0; k < kMfUnroll; ++k) acc[k] = T(0);
          const TS* p = panel + d.panel;
          int i = j + lane;
          for (; i + 32 < d.ns; i += 64) {      // two rows per lane in flight
            T x[kMfUnroll], x2[kMfUnroll];
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) {
              const bool c = j + k < jend;
              x[k] = (c && i >= j + k) ? T(ld_f(p + mf_cofs(nf, j + k) + i)) : T(0);
              x2[k] = c ? T(ld_f(p + mf_cofs(nf, j + k) + i + 32)) : T(0);
            }
            const T gi = g[i], gi2 = g[i + 32];
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) acc[k] += x[k] * gi + x2[k] * gi2;
          }
          if (i < d.ns) {
            T x[kMfUnroll];
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) x[k] = (j + k < jend && i >= j + k) ? T(ld_f(p + mf_cofs(nf, j + k) + i)) : T(0);
            const T gi = g[i];
#pragma unroll
            for (int k = 0; k < kMfUnroll; ++k) acc[k] += x[k] * gi;
          }
#pragma unroll
          for (int k = 0; k < kMfUnroll; ++k) {
            const T sum = warp_sum(acc[k]);
            if (lane == 0 && j + k < jend) stage[d.stage + j + k] = sum;
          }
        }
      }
      __syncthreads();
      for (int t = L.br + tid; t < E.br; t += nt) v[a.brows[t]] = stage[t - L.br];
    }
    __syncthreads();
  }
  for (int p = tid; p < m; p += nt) zloc[base + a.nd_loc[base + p]] = v[p];
}

MfSolveArgs solve_args(const Ctx* c) {
  MfSolveArgs a;
  a.om_ptr = c->om_ptr;
  a.sub_lv = c->mf_sub_lv;
  a.sub_panel = c->mf_sub_panel;
  a.sub_brow = c->mf_sub_brow;
  a.lv = c->mf_lv;
  a.rows = c->mf_rows;
  a.brows = c->mf_brows;
  a.st = c->mf_st;
  a.xt = c->mf_xt;
  a.ut = c->mf_ut;
  a.nd_dof = c->mf_nd_dof;
  a.nd_loc = c->mf_nd_loc;
  a.pullS_ptr = c->mf_pullS_ptr;
  a.pullB_ptr = c->mf_pullB_ptr;
  a.pullS = c->mf_pullS;
  a.pullB = c->mf_pullB;
  a.bidx = c->mf_bidx;
  a.arena = c->mf_arena;
  a.vlen = (c->max_m + 3) & ~3;
  a.stage = c->mf_stage;
  a.err = c->derr;
  a.wait_cycles = c->wait_cycles > 0 ? c->wait_cycles : kDefaultWaitCycles;
  return a;
}

// Shared memory of the solve: the warps' barriers, the local vector, the
// large supernodes' stage and one panel buffer per warp.
size_t solve_smem(const Ctx* c, size_t es) {
  return 64 * sizeof(uint64_t) + size_t((c->max_m + 3) & ~3) * es + size_t(c->mf_stage) * es +
         size_t(c->mf_threads / 32) * mf_buf_bytes(int(es));
}

}  // namespace

gdsw_status mf_configure(Ctx* c) {
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  if (solve_smem(c, es) > size_t(max_block_smem_optin())) {
    set_error("subdomain of %d unknowns does not fit the multifrontal solve's shared memory", c->max_m);
    return GDSW_ERR_UNSUPPORTED;
  }
  if (c->fp16) GDSW_CK(allow_max_dynamic_smem(k_local_mf<float, __half>));
  else if (c->fp32) GDSW_CK(allow_max_dynamic_smem(k_local_mf<float, float>));
  else GDSW_CK(allow_max_dynamic_smem(k_local_mf<double, double>));
  return GDSW_OK;
}

// Panels are stored in FP16 (FP16 precision), FP32 or FP64; the solve
// computes in FP32 or FP64.
gdsw_status mf_launch_local(Ctx* c, const double* r, cudaStream_t s, const KrylovScalars* ks) {
  const MfSolveArgs a = solve_args(c);
  if (c->fp16) {
    k_local_mf<float, __half><<<c->nsub, c->mf_threads, solve_smem(c, sizeof(float)), s>>>(
        r, a, static_cast<const __half*>(c->mf_panel), static_cast<float*>(c->mf_arena_buf),
        static_cast<float*>(c->zloc), ks);
  } else if (c->fp32) {
    k_local_mf<float, float><<<c->nsub, c->mf_threads, solve_smem(c, sizeof(float)), s>>>(
        r, a, static_cast<const float*>(c->mf_panel), static_cast<float*>(c->mf_arena_buf),
        static_cast<float*>(c->zloc), ks);
  } else {
    k_local_mf<double, double><<<c->nsub, c->mf_threads, solve_smem(c, sizeof(double)), s>>>(
        r, a, static_cast<const double*>(c->mf_panel), static_cast<double*>(c->mf_arena_buf),
        static_cast<double*>(c->zloc), ks);
  }
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

gdsw_status mf_numeric_setup(Ctx* c, const Plan& P, const double* d_araw, cudaStream_t s) {
  const bool f32 = c->fp32, f16 = c->fp16;
  const size_t es = f32 ? sizeof(float) : sizeof(double);     // vectors
  const size_t ps = f16 ? sizeof(__half) : es;                // panels
  // the plan depends on the pattern alone: a refactor reuses the setup's
  if (!c->mf_plan_host) {
    auto plan = std::make_shared<MfPlan>();
    GDSW_TRY(build_mf_plan(P, mf_leaf_size(), mf_buf_bytes(int(es)) / int(ps), plan.get()));
    c->mf_plan_host = std::move(plan);
  }
  const MfPlan& M = *c->mf_plan_host;
  // resident solve data
  GDSW_TRY(upload(c, &c->mf_sn, M.sn, s));
  GDSW_TRY(upload(c, &c->mf_sub_panel, M.sub_panel, s));
  GDSW_TRY(upload(c, &c->mf_sub_brow, M.sub_brow, s));
  GDSW_TRY(upload(c, &c->mf_st, M.stasks, s));
  GDSW_TRY(upload(c, &c->mf_brows, M.brows, s));
  GDSW_TRY(upload(c, &c->mf_sub_sn, M.sub_sn, s));
  GDSW_TRY(upload(c, &c->mf_sub_lv, M.sub_lv, s));
  GDSW_TRY(upload(c, &c->mf_lv, M.lv, s));
  GDSW_TRY(upload(c, &c->mf_rows, M.rows, s));
  GDSW_TRY(upload(c, &c->mf_xt, M.xtasks, s));
  GDSW_TRY(upload(c, &c->mf_ut, M.utasks, s));
  GDSW_TRY(upload(c, &c->mf_nd_dof, M.nd_dof, s));
  GDSW_TRY(upload(c, &c->mf_nd_loc, M.nd_loc, s));
  GDSW_TRY(upload(c, &c->mf_pullS_ptr, M.pullS_ptr, s));
  GDSW_TRY(upload(c, &c->mf_pullB_ptr, M.pullB_ptr, s));
  GDSW_TRY(upload(c, &c->mf_pullS, M.pullS_ent, s));
  GDSW_TRY(upload(c, &c->mf_pullB, M.pullB_ent, s));
  GDSW_TRY(upload(c, &c->mf_bidx, M.bidx, s));
  c->mf_arena = std::max(1, M.arena_max);
  c->mf_stage = (M.stage_max + 3) & ~3;
  if (f16) {
    __half* p;
    GDSW_TRY(dalloc(c, &p, size_t(M.panel_total)));
    c->mf_panel = p;
  } else if (f32) {
    float* p;
    GDSW_TRY(dalloc(c, &p, size_t(M.panel_total)));
    c->mf_panel = p;
  } else {
    double* p;
    GDSW_TRY(dalloc(c, &p, size_t(M.panel_total)));
    c->mf_panel = p;
  }
  if (f32) {
    float* ar;
    GDSW_TRY(dalloc(c, &ar, size_t(c->nsub) * c->mf_arena));
    c->mf_arena_buf = ar;
  } else {
    double* ar;
    GDSW_TRY(dalloc(c, &ar, size_t(c->nsub) * c->mf_arena));
    c->mf_arena_buf = ar;
  }
  GDSW_CK(cudaMemsetAsync(c->mf_panel, 0, size_t(M.panel_total) * ps, s));

  // factorisation, in batches of subdomains whose work areas fit the budget
  struct Tmp {
    std::vector<void*> p;
    ~Tmp() { for (void* q : p) cudaFree(q); }
    gdsw_status get(void** out, size_t bytes) {
      *out = nullptr;
      if (cudaMalloc(out, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu scratch bytes failed", bytes);
        return GDSW_ERR_OUT_OF_MEMORY;
      }
      p.push_back(*out);
      return GDSW_OK;
    }
  } tmp;
  auto put = [&](const void* src, size_t bytes, cudaStream_t st) -> void* {
    void* q = nullptr;
    if (tmp.get(&q, bytes) != GDSW_OK) return nullptr;
    if (bytes && cudaMemcpyAsync(q, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    return q;
  };
  MfFactorArgs fa{};
  fa.ch_ptr = static_cast<const int*>(put(M.ch_ptr.data(), M.ch_ptr.size() * 4, s));
  fa.ch_list = static_cast<const int*>(put(M.ch_list.data(), M.ch_list.size() * 4, s));
  fa.relF = static_cast<const uint16_t*>(put(M.relF.data(), M.relF.size() * 2, s));
  fa.asm_ptr = static_cast<const int*>(put(M.asm_ptr.data(), M.asm_ptr.size() * 4, s));
  fa.asm_ent = static_cast<const int*>(put(M.asm_ent.data(), M.asm_ent.size() * 4, s));
  fa.asm_rc = static_cast<const uint32_t*>(put(M.asm_rc.data(), M.asm_rc.size() * 4, s));
  fa.stack_off = static_cast<const int64_t*>(put(M.stack_off.data(), M.stack_off.size() * 8, s));
  void* p = nullptr;
  GDSW_TRY(tmp.get(&p, 4));
  fa.err = static_cast<int*>(p);
  if (!fa.ch_ptr || !fa.ch_list || !fa.relF || !fa.asm_ptr || !fa.asm_ent || !fa.asm_rc || !fa.stack_off) {
    set_error("multifrontal setup: scratch allocation or copy failed");
    return GDSW_ERR_OUT_OF_MEMORY;
  }
  GDSW_CK(cudaMemsetAsync(fa.err, 0, 4, s));
  fa.sn = c->mf_sn;
  fa.sub_sn = c->mf_sub_sn;
  fa.araw = d_araw;
  fa.front_len = int64_t(M.max_front) * M.max_front;
  fa.inv_len = int64_t(M.max_ns) * M.max_ns;
  const int nsub = P.nsub;
  std::vector<std::pair<int, int>> batches;
  const int64_t cap = mf_batches(M, nsub, &batches);
  GDSW_TRY(tmp.get(&p, size_t(cap) * 8));
  fa.work = static_cast<double*>(p);
  GDSW_TRY(tmp.get(&p, size_t(nsub) * 8));
  int64_t* d_off = static_cast<int64_t*>(p);
  fa.work_off = d_off;
  const size_t shm = size_t(std::max(1, M.max_front)) * sizeof(double);
  if (shm > size_t(max_block_smem_optin())) { set_error("front of %d rows too large", M.max_front); return GDSW_ERR_UNSUPPORTED; }
  if (f16) GDSW_CK(allow_max_dynamic_smem(k_mf_factor<__half>));
  else if (f32) GDSW_CK(allow_max_dynamic_smem(k_mf_factor<float>));
  else GDSW_CK(allow_max_dynamic_smem(k_mf_factor<double>));
  std::vector<int64_t> off;
  for (const auto& b : batches) {
    off.clear();
    int64_t tot = 0;
    for (int q = b.first; q < b.second; ++q) { off.push_back(tot); tot += mf_work_need(M, q); }
    GDSW_CK(cudaMemcpyAsync(d_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s));
    fa.q0 = b.first;
    if (f16) k_mf_factor<__half><<<b.second - b.first, 512, shm, s>>>(fa, static_cast<__half*>(c->mf_panel));
    else if (f32) k_mf_factor<float><<<b.second - b.first, 512, shm, s>>>(fa, static_cast<float*>(c->mf_panel));
    else k_mf_factor<double><<<b.second - b.first, 512, shm, s>>>(fa, static_cast<double*>(c->mf_panel));
    GDSW_CK(cudaGetLastError());
    GDSW_CK(cudaStreamSynchronize(s));   // the work areas and offsets are reused by the next batch
  }
  int h = 0;
  GDSW_CK(cudaMemcpyAsync(&h, fa.err, 4, cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (h & MF_ERR_BREAKDOWN) {
    set_error("exact local factorisation: non-positive pivot (A_s not SPD)");
    return GDSW_ERR_BREAKDOWN;
  }
  c->mf = true;
  c->stats.dense_local = M.panel_total;
  c->stats.mf_supernodes = static_cast<int64_t>(M.sn.size());
  c->stats.mf_levels = static_cast<int64_t>(M.lv.size()) - 1;
  return mf_configure(c);
}

}  // namespace gdsw
