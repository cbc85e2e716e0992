// Numeric setup on the device (Sec. V-A1 (b)): local matrices and their
// incomplete factors by fixed-point sweeps (Sec. V-B3), the GDSW basis
// (Sec. III, Eq. 2), the coarse matrix A0 = Phi^T A Phi and its inverse, and
// the dense inverses of the exact local solver.
//
// B300 FP64 runs on CUDA cores (no fast FP64 tensor path on this part), so the
// dense kernels here are plain FP64 loops organised for L2 reuse; they run
// once per setup and are not on the per-iteration path.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace gdsw {

namespace {

constexpr double kDropTol = 1e-10;   // relative norm below which an MGS column is dropped

enum { ERR_BREAKDOWN = 1 };

// ---------------------------------------------------------------------------
// local matrices: values, symmetric unit-diagonal scaling
// ---------------------------------------------------------------------------

// One CTA per subdomain: s_i = a_ii^-1/2 for every local row, then
// a~_e = a_e s_i s_j (Chow-Patel scaling) and the raw value a_e.
__global__ void k_extract_local(const double* __restrict__ val, const int* __restrict__ om_ptr,
                                const int* __restrict__ lm_sub_ent, const int* __restrict__ lm_gent,
                                const uint16_t* __restrict__ lm_row, const int* __restrict__ lm_col,
                                const int* __restrict__ lm_diag, double* __restrict__ sc,
                                double* __restrict__ at, double* __restrict__ araw, int* err) {
  const int s = blockIdx.x;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double d = val[lm_gent[lm_diag[base + i]]];
    if (!(d > 0.0)) { atomicOr(err, ERR_BREAKDOWN); sc[base + i] = 1.0; }
    else sc[base + i] = 1.0 / sqrt(d);
  }
  __syncthreads();
  for (int e = lm_sub_ent[s] + threadIdx.x; e < lm_sub_ent[s + 1]; e += blockDim.x) {
    const int g = lm_gent[e];
    const double a = g >= 0 ? val[g] : 0.0;      // fill of IC(k)/ILU(k) starts at zero
    araw[e] = a;
    at[e] = a * sc[base + lm_row[e]] * sc[base + lm_col[e]];
  }
}

// One synchronous IC(0) sweep (Sec. V-B3) over every lower entry of every
// subdomain (one thread per entry; one launch per sweep, so every entry of
// sweep k+1 reads sweep-k values):
//   s_ij = a~_ij - sum_{k<j} l_ik l_jk;  l_ij = s_ij / l_jj (i>j),  l_jj = sqrt(s_jj).
// The sum merges row i and row j of the local pattern over columns k < j.
__global__ void k_ic0_sweep(int nent, const int* __restrict__ ebase, const int* __restrict__ lm_rowptr,
                            const int* __restrict__ lm_col, const uint16_t* __restrict__ lm_row,
                            const int* __restrict__ lm_diag, const double* __restrict__ at,
                            const double* __restrict__ Fo, double* __restrict__ Fn, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
    const int base = ebase[e];
    const int i = lm_row[e], j = lm_col[e];
    if (j > i) { Fn[e] = Fo[e]; continue; }
    int a = lm_rowptr[base + i];
    const int ae = lm_rowptr[base + i + 1];
    int b = lm_rowptr[base + j];
    const int be = lm_diag[base + j];
    double acc = 0.0;
    while (a < ae && b < be) {
      const int ca = lm_col[a], cb = lm_col[b];
      if (ca >= j) break;
      if (ca == cb) { acc = fma(Fo[a], Fo[b], acc); ++a; ++b; }
      else if (ca < cb) ++a;
      else ++b;
    }
    const double sv = at[e] - acc;
    if (i == j) {
      if (!(sv > 0.0)) { atomicOr(err, ERR_BREAKDOWN); Fn[e] = 1.0; }
      else Fn[e] = sqrt(sv);
    } else {
      Fn[e] = sv / Fo[lm_diag[base + j]];
    }
  }
}

// One synchronous ILU(0) sweep over the full pattern (L unit lower, U upper):
//   l_ij = (a~_ij - sum_{k<j} l_ik u_kj) / u_jj  (i>j),   u_ij = a~_ij - sum_{k<i} l_ik u_kj.
// u_kj is read from the entry (k, j) reached through the transposed position of (j, k).
__global__ void k_ilu0_sweep(int nent, const int* __restrict__ ebase, const int* __restrict__ lm_rowptr,
                             const int* __restrict__ lm_col, const uint16_t* __restrict__ lm_row,
                             const int* __restrict__ lm_diag, const int* __restrict__ lm_tpos,
                             const double* __restrict__ at, const double* __restrict__ Fo,
                             double* __restrict__ Fn, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
    const int base = ebase[e];
    const int i = lm_row[e], j = lm_col[e];
    const int kmax = min(i, j);
    int a = lm_rowptr[base + i];
    const int ae = lm_rowptr[base + i + 1];
    int b = lm_rowptr[base + j];
    const int be = lm_rowptr[base + j + 1];
    double acc = 0.0;
    while (a < ae && b < be) {
      const int ca = lm_col[a], cb = lm_col[b];
      if (ca >= kmax || cb >= kmax) break;
      if (ca == cb) { acc = fma(Fo[a], Fo[lm_tpos[b]], acc); ++a; ++b; }
      else if (ca < cb) ++a;
      else ++b;
    }
    const double sv = at[e] - acc;
    if (i > j) {
      const double u = Fo[lm_diag[base + j]];
      if (u == 0.0) { atomicOr(err, ERR_BREAKDOWN); Fn[e] = 0.0; }
      else Fn[e] = sv / u;
    } else {
      Fn[e] = sv;
    }
  }
}

// Undo the scaling entry by entry: the factors of A_s itself.
// IC:  L^ = S^-1 L  (l^_ij = l_ij / s_i).
// ILU: L^ = S^-1 L S (l^_ij = l_ij s_j / s_i), U^ = S^-1 U S^-1 (u^_ij = u_ij / (s_i s_j)).
__global__ void k_unscale(int nent, int ilu, const int* __restrict__ lm_row_abs_base,
                          const uint16_t* __restrict__ lm_row, const int* __restrict__ lm_col,
                          const int* __restrict__ ent_sub_base, const double* __restrict__ sc,
                          const double* __restrict__ F, double* __restrict__ G) {
  (void)lm_row_abs_base;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
    const int base = ent_sub_base[e];
    const double si = sc[base + lm_row[e]], sj = sc[base + lm_col[e]];
    const int i = lm_row[e], j = lm_col[e];
    double g;
    if (!ilu) g = (j <= i) ? F[e] / si : 0.0;
    else g = (j < i) ? F[e] * sj / si : F[e] / (si * sj);
    G[e] = g;
  }
}

template <class T>
__global__ void k_pack_ell(int64_t nslots, const int* __restrict__ src, const double* __restrict__ G,
                           T* __restrict__ val) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nslots;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int e = src[q];
    val[q] = e >= 0 ? T(G[e]) : T(0);
  }
}

template <class T>
__global__ void k_pack_dinv(int64_t nrows, const int* __restrict__ dsrc, const double* __restrict__ G,
                            T* __restrict__ dinv) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nrows;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int e = dsrc[q];
    dinv[q] = e >= 0 ? T(1.0 / G[e]) : T(1);
  }
}

// Values of the per-level record stream (see build_records): slot q of the
// level-sliced ELL goes to element valpos[q] of the stream, the inverse
// diagonal of level-ordered row i to element dinvpos[i].
template <class T>
__device__ __forceinline__ T from_double(double v) { return T(v); }
template <>
__device__ __forceinline__ __half from_double<__half>(double v) { return __double2half(v); }

template <class T>
__global__ void k_fill_records(int64_t nslots, const int* __restrict__ src,
                               const uint32_t* __restrict__ valpos, int64_t nrows,
                               const int* __restrict__ dsrc, const uint32_t* __restrict__ dinvpos,
                               const double* __restrict__ G, T* __restrict__ stream) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nslots; q += stride) {
    const int e = src[q];
    stream[valpos[q]] = from_double<T>(e >= 0 ? G[e] : 0.0);
  }
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nrows; q += stride) {
    const int e = dsrc[q];
    stream[dinvpos[q]] = from_double<T>(e >= 0 ? 1.0 / G[e] : 1.0);
  }
}

// ---------------------------------------------------------------------------
// Phi_Gamma: orthonormal basis of the null space on each component
// ---------------------------------------------------------------------------

// One CTA per coarse-space owner: modified Gram-Schmidt over the nn columns of
// the null space restricted to the owner's support and scaled by the support
// weights, in column order, dropping a column whose remaining norm is below
// kDropTol of its original norm.  Kept column k of owner o sits at
// Q[supp_ptr[o]*nn + k*R + r]; rank[o] counts the kept columns.
__global__ void k_mgs(const int* __restrict__ supp_ptr, const int* __restrict__ supp_dof,
                      const double* __restrict__ supp_w, const double* __restrict__ Z, int n, int nn,
                      double* __restrict__ Q, int* __restrict__ rank) {
  __shared__ double sh[32];
  __shared__ double bc;
  const int o = blockIdx.x;
  const int r0 = supp_ptr[o], R = supp_ptr[o + 1] - r0;
  double* Qc = Q + int64_t(r0) * nn;
  int kept = 0;
  for (int col = 0; col < nn; ++col) {
    double* v = Qc + int64_t(kept) * R;
    double loc = 0.0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const double z = Z[int64_t(col) * n + supp_dof[r0 + r]] * supp_w[r0 + r];
      v[r] = z;
      loc += z * z;
    }
    double t = block_sum(loc, sh);
    if (threadIdx.x == 0) bc = sqrt(t);
    __syncthreads();
    const double n0 = bc;
    __syncthreads();
    for (int k = 0; k < kept; ++k) {
      const double* qk = Qc + int64_t(k) * R;
      loc = 0.0;
      for (int r = threadIdx.x; r < R; r += blockDim.x) loc += qk[r] * v[r];
      t = block_sum(loc, sh);
      if (threadIdx.x == 0) bc = t;
      __syncthreads();
      const double d = bc;
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) v[r] -= d * qk[r];
      __syncthreads();
    }
    loc = 0.0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) loc += v[r] * v[r];
    t = block_sum(loc, sh);
    if (threadIdx.x == 0) bc = sqrt(t);
    __syncthreads();
    const double nv = bc;
    __syncthreads();
    if (n0 == 0.0 || nv < kDropTol * n0) continue;
    const double inv = 1.0 / nv;
    for (int r = threadIdx.x; r < R; r += blockDim.x) v[r] *= inv;
    __syncthreads();
    ++kept;
  }
  if (threadIdx.x == 0) rank[o] = kept;
}

// Scatter each owner's kept columns into the interface-component blocks of Phi
// (column-major): support entry e lies in component supp_comp[e], row
// supp_row[e], and the owner's columns start at supp_colpos[e] in that block.
__global__ void k_copy_phig(int nsub, const int* __restrict__ supp_ptr,
                            const int* __restrict__ supp_comp, const int* __restrict__ supp_row,
                            const int* __restrict__ supp_colpos, const int* __restrict__ owner_k,
                            int nn, const double* __restrict__ Q, const int* __restrict__ brow_ptr,
                            const int64_t* __restrict__ phi_off, double* __restrict__ phi) {
  const int o = blockIdx.x;
  const int r0 = supp_ptr[o], R = supp_ptr[o + 1] - r0;
  const int k = owner_k[o];
  const double* Qc = Q + int64_t(r0) * nn;
  for (int q = threadIdx.x; q < R * k; q += blockDim.x) {
    const int t = q / R, e = q - t * R;
    const int b = nsub + supp_comp[r0 + e];
    const int nr = brow_ptr[b + 1] - brow_ptr[b];
    phi[phi_off[b] + int64_t(supp_colpos[r0 + e] + t) * nr + supp_row[r0 + e]] = Qc[q];
  }
}

// ---------------------------------------------------------------------------
// Banded Cholesky (natural order) for A_IsIs (Eq. 2) and the exact solver
// ---------------------------------------------------------------------------
// Band storage, lower triangle, column-major: entry (i, j), 0 <= i-j <= w, at
// j*(w+1) + (i-j).  One CTA per matrix; right-looking, one column at a time,
// the pivot column staged in shared memory.
__global__ void k_band_cholesky(double* band, const int64_t* __restrict__ boff,
                                const int* __restrict__ bn, const int* __restrict__ bw, int p0,
                                int* err) {
  extern __shared__ double colv[];
  const int p = p0 + blockIdx.x;
  double* B = band + boff[p];
  const int n = bn[p], w = bw[p], W = w + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    double* Bj = B + int64_t(j) * W;
    if (threadIdx.x == 0) {
      const double d = Bj[0];
      if (!(d > 0.0)) { atomicOr(err, ERR_BREAKDOWN); piv = 1.0; }
      else piv = sqrt(d);
      Bj[0] = piv;
    }
    __syncthreads();
    const int len = min(w, n - 1 - j);
    const double ip = 1.0 / piv;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      const double v = Bj[1 + t] * ip;
      Bj[1 + t] = v;
      colv[t] = v;
    }
    __syncthreads();
    // trailing update of the (len x len) lower triangle: column kk of the
    // window is column j+1+kk of the band
    for (int kk = wid; kk < len; kk += nw) {
      double* Bk = B + int64_t(j + 1 + kk) * W;
      const double lk = colv[kk];
      for (int ii = kk + lane; ii < len; ii += 32) Bk[ii - kk] -= colv[ii] * lk;
    }
    __syncthreads();
  }
}

// Solve (L L^T) X = RHS in place for a column-major RHS of k columns
// (leading dimension n) with the band factor.  Forward: right-looking with
// the factor column; backward: dot products with the factor column.
__global__ void k_band_solve(const double* __restrict__ band, const int64_t* __restrict__ boff,
                             const int* __restrict__ bn, const int* __restrict__ bw,
                             double* rhs, const int64_t* __restrict__ roff,
                             const int* __restrict__ rk, int p0) {
  __shared__ double sh[32];
  const int p = p0 + blockIdx.x;
  const double* B = band + boff[p];
  const int n = bn[p], w = bw[p], W = w + 1, k = rk[p];
  double* X = rhs + roff[p];
  if (k == 0 || n == 0) return;
  // forward: x_j /= l_jj; x_i -= l_ij x_j for i in (j, j+w]
  for (int j = 0; j < n; ++j) {
    const double* Bj = B + int64_t(j) * W;
    const int len = min(w, n - 1 - j);
    const double ip = 1.0 / Bj[0];
    __syncthreads();
    // every thread computes x_j for the columns it touches (reads before any write)
    for (int q = threadIdx.x; q < len * k; q += blockDim.x) {
      const int c = q / len, t = q - c * len;
      const double xj = X[int64_t(c) * n + j] * ip;
      X[int64_t(c) * n + j + 1 + t] -= Bj[1 + t] * xj;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) X[int64_t(c) * n + j] *= ip;
  }
  __syncthreads();
  // backward: x_j = (x_j - sum_{i>j} l_ij x_i) / l_jj
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = n - 1; j >= 0; --j) {
    const double* Bj = B + int64_t(j) * W;
    const int len = min(w, n - 1 - j);
    for (int c = wid; c < k; c += nw) {
      double* Xc = X + int64_t(c) * n;
      double acc = 0.0;
      for (int t = lane; t < len; t += 32) acc += Bj[1 + t] * Xc[j + 1 + t];
      acc = warp_sum(acc);
      if (lane == 0) Xc[j] = (Xc[j] - acc) / Bj[0];
    }
    __syncthreads();
  }
  (void)sh;
}

// Interior blocks: band of A_IsIs and the right-hand sides -A_IsGamma Phi_Gamma
// written straight into the interior block of Phi (zeroed beforehand).
__global__ void k_assemble_interior(int s0, const int* __restrict__ rowptr,
                                    const int* __restrict__ colind, const double* __restrict__ val,
                                    const int* __restrict__ int_ptr, const int* __restrict__ int_dofs,
                                    const int* __restrict__ dof_comp,
                                    const int* __restrict__ dof_comprow,
                                    const int* __restrict__ dof_introw,
                                    int nsub, const int* __restrict__ brow_ptr,
                                    const int* __restrict__ bcol_ptr, const int* __restrict__ bcol,
                                    const int64_t* __restrict__ phi_off, double* __restrict__ phi,
                                    double* band, const int64_t* __restrict__ boff,
                                    const int* __restrict__ bw) {
  const int s = s0 + blockIdx.x;
  const int ns = int_ptr[s + 1] - int_ptr[s];
  const int W = bw[s] + 1;
  double* B = band + boff[s];
  double* Ph = phi + phi_off[s];
  const int* cols = bcol + bcol_ptr[s];
  const int ncols = bcol_ptr[s + 1] - bcol_ptr[s];
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const int g = int_dofs[int_ptr[s] + i];
    for (int e = rowptr[g]; e < rowptr[g + 1]; ++e) {
      const int c = colind[e];
      const int comp = dof_comp[c];
      if (comp < 0) {
        const int j = dof_introw[c];
        if (j <= i) B[int64_t(j) * W + (i - j)] = val[e];
        continue;
      }
      const int b = nsub + comp;
      const int kc = bcol_ptr[b + 1] - bcol_ptr[b];
      if (kc == 0) continue;
      const int Rc = brow_ptr[b + 1] - brow_ptr[b];
      const double* Pc = phi + phi_off[b];
      const int rr = dof_comprow[c];
      const int* ccols = bcol + bcol_ptr[b];
      for (int t = 0; t < kc; ++t) {
        // position of the component's column in the interior block's sorted list
        const int l = ccols[t];
        int lo = 0, hi = ncols;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (cols[mid] < l) lo = mid + 1; else hi = mid; }
        Ph[int64_t(lo) * ns + i] -= val[e] * Pc[int64_t(t) * Rc + rr];
      }
    }
  }
}

// Band of A_s (exact local solver) from the local CSR values.
__global__ void k_assemble_local_band(const int* __restrict__ om_ptr, const int* __restrict__ lm_sub_ent,
                                      const uint16_t* __restrict__ lm_row, const int* __restrict__ lm_col,
                                      const double* __restrict__ araw, double* band,
                                      const int64_t* __restrict__ boff, const int* __restrict__ bw,
                                      int p0) {
  const int s = p0 + blockIdx.x;
  const int W = bw[s] + 1;
  double* B = band + boff[s];
  for (int e = lm_sub_ent[s] + threadIdx.x; e < lm_sub_ent[s + 1]; e += blockDim.x) {
    const int i = lm_row[e], j = lm_col[e];
    if (j <= i) B[int64_t(j) * W + (i - j)] = araw[e];
  }
}

__global__ void k_set_identity(double* X, const int64_t* __restrict__ xoff, const int* __restrict__ xn,
                               int p0) {
  const int p = p0 + blockIdx.x;
  const int n = xn[p];
  double* Xp = X + xoff[p];
  for (int i = threadIdx.x; i < n; i += blockDim.x) Xp[int64_t(i) * n + i] = 1.0;
}

template <class T>
__global__ void k_convert(int64_t len, const double* __restrict__ a, T* __restrict__ b) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < len;
       q += int64_t(gridDim.x) * blockDim.x)
    b[q] = T(a[q]);
}

// ---------------------------------------------------------------------------
// Coarse matrix A0 = Phi^T A Phi = Phi_Gamma^T (A Phi)_Gamma  ((A Phi)_I = 0 by Eq. 2)
// ---------------------------------------------------------------------------
// One CTA (one warp) per coarse row k, whose function lives on its owner's support:
//   A0[k, :] = sum_{g in supp(k)} Phi[g, k] sum_j A[g, j] Phi[j, :]
// accumulated in shared memory in a fixed order (deterministic).
__global__ void k_coarse_rows(int nsub, const int* __restrict__ coarse_owner,
                              const int* __restrict__ owner_c0, const int* __restrict__ coarse_prob,
                              const int* __restrict__ prob_c0, const int64_t* __restrict__ a0_off,
                              const int* __restrict__ rowptr,
                              const int* __restrict__ colind, const double* __restrict__ val,
                              const int* __restrict__ brow_ptr, const int* __restrict__ supp_ptr,
                              const int* __restrict__ supp_dof, const int* __restrict__ supp_comp,
                              const int* __restrict__ supp_row, const int* __restrict__ supp_colpos,
                              const int* __restrict__ bcol_ptr, const int* __restrict__ bcol,
                              const int64_t* __restrict__ phi_off, const double* __restrict__ phi,
                              const int* __restrict__ dof_blk, const int* __restrict__ dof_blkrow,
                              double* __restrict__ A0) {
  extern __shared__ double acc[];
  const int k = blockIdx.x;
  const int o = coarse_owner[k];                  // owner index (support range)
  const int t = k - owner_c0[o];
  const int pr = coarse_prob[k];
  const int cp = prob_c0[pr], np = prob_c0[pr + 1] - cp;   // this problem's coarse block
  for (int l = threadIdx.x; l < np; l += blockDim.x) acc[l] = 0.0;
  __syncwarp();
  for (int sidx = supp_ptr[o]; sidx < supp_ptr[o + 1]; ++sidx) {
    const int g = supp_dof[sidx];
    const int b = nsub + supp_comp[sidx];
    const int R = brow_ptr[b + 1] - brow_ptr[b];
    const double pk = phi[phi_off[b] + int64_t(supp_colpos[sidx] + t) * R + supp_row[sidx]];
    for (int e = rowptr[g]; e < rowptr[g + 1]; ++e) {
      const int j = colind[e];
      const double coef = pk * val[e];
      const int bj = dof_blk[j], rj = dof_blkrow[j];
      const int nr = brow_ptr[bj + 1] - brow_ptr[bj];
      const int c0 = bcol_ptr[bj], kc = bcol_ptr[bj + 1] - c0;
      const double* Pj = phi + phi_off[bj] + rj;
      for (int u = threadIdx.x; u < kc; u += 32) acc[bcol[c0 + u] - cp] += coef * Pj[int64_t(u) * nr];
      __syncwarp();
    }
  }
  double* row = A0 + a0_off[pr] + int64_t(k - cp) * np;
  for (int l = threadIdx.x; l < np; l += blockDim.x) row[l] = acc[l];
}

// ---------------------------------------------------------------------------
// Dense FP64 Cholesky of A0 (row-major, lower, tiles of 32) and A0^-1
// ---------------------------------------------------------------------------
constexpr int NB = 32;

__global__ void k_potrf_diag(double* A, int n, int J, int* err) {
  __shared__ double T[NB][NB + 1];
  const int j0 = J * NB, nb = min(NB, n - j0);
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int r = q / NB, c = q % NB;
    T[r][c] = (r < nb && c < nb) ? A[int64_t(j0 + r) * n + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (threadIdx.x == 0) {
      const double d = T[c][c];
      if (!(d > 0.0)) { atomicOr(err, ERR_BREAKDOWN); T[c][c] = 1.0; }
      else T[c][c] = sqrt(d);
    }
    __syncthreads();
    const double ip = 1.0 / T[c][c];
    for (int r = c + 1 + threadIdx.x; r < nb; r += blockDim.x) T[r][c] *= ip;
    __syncthreads();
    for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
      const int r = q / NB, cc = q % NB;
      if (cc > c && r >= cc && r < nb) T[r][cc] -= T[r][c] * T[cc][c];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int r = q / NB, c = q % NB;
    if (r < nb && c <= r) A[int64_t(j0 + r) * n + j0 + c] = T[r][c];
  }
}

// L_IJ = A_IJ L_JJ^-T for every row tile I > J (one CTA per tile, thread per row).
__global__ void k_trsm_panel(double* A, int n, int J) {
  __shared__ double Ld[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int j0 = J * NB, nb = min(NB, n - j0);
  const int i0 = (J + 1 + blockIdx.x) * NB, mb = min(NB, n - i0);
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int r = q / NB, c = q % NB;
    Ld[r][c] = (r < nb && c < nb) ? A[int64_t(j0 + r) * n + j0 + c] : 0.0;
    X[r][c] = (r < mb && c < nb) ? A[int64_t(i0 + r) * n + j0 + c] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (r < mb) {
    for (int c = 0; c < nb; ++c) {
      double v = X[r][c];
      for (int k = 0; k < c; ++k) v -= X[r][k] * Ld[c][k];
      X[r][c] = v / Ld[c][c];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int rr = q / NB, c = q % NB;
    if (rr < mb && c < nb) A[int64_t(i0 + rr) * n + j0 + c] = X[rr][c];
  }
}

// A_IK -= L_IJ L_KJ^T for J < K <= I (grid over (I, K) tile pairs of the trailing part).
__global__ void k_syrk_update(double* A, int n, int J) {
  const int I = J + 1 + blockIdx.y, K = J + 1 + blockIdx.x;
  if (K > I) return;
  __shared__ double Li[NB][NB + 1];
  __shared__ double Lk[NB][NB + 1];
  const int j0 = J * NB, nb = min(NB, n - j0);
  const int i0 = I * NB, k0 = K * NB;
  const int mi = min(NB, n - i0), mk = min(NB, n - k0);
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int r = q / NB, c = q % NB;
    Li[r][c] = (r < mi && c < nb) ? A[int64_t(i0 + r) * n + j0 + c] : 0.0;
    Lk[r][c] = (r < mk && c < nb) ? A[int64_t(k0 + r) * n + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
    const int r = q / NB, c = q % NB;
    if (r >= mi || c >= mk) continue;
    if (I == K && c > r) continue;
    double v = 0.0;
#pragma unroll 8
    for (int t = 0; t < NB; ++t) v += Li[r][t] * Lk[c][t];
    A[int64_t(i0 + r) * n + k0 + c] -= v;
  }
}

// Columns [32*blockIdx.x, +32) of A0^-1 from the Cholesky factor: forward
// L Y = E then backward L^T X = Y.  Thread (c, part): column c, every 8th
// term of each inner product; parts are summed in a fixed order.
__global__ void k_chol_inverse(const double* __restrict__ L, int n, double* W, double* Ainv) {
  __shared__ double red[8][NB + 1];
  const int c = threadIdx.x & 31, part = threadIdx.x >> 5;
  const int col = blockIdx.x * NB + c;
  const bool active = col < n;
  double* Y = W + int64_t(blockIdx.x) * NB * n;   // Y[c*n + r]
  const int cstart = blockIdx.x * NB;
  for (int r = part; r < n; r += 8)
    if (active) Y[int64_t(c) * n + r] = 0.0;
  __syncthreads();
  for (int r = cstart; r < n; ++r) {
    double acc = 0.0;
    if (active)
      for (int k = cstart + part; k < r; k += 8) acc += L[int64_t(r) * n + k] * Y[int64_t(c) * n + k];
    red[part][c] = acc;
    __syncthreads();
    if (part == 0 && active) {
      double s = 0.0;
      for (int q = 0; q < 8; ++q) s += red[q][c];
      const double e = (r == col) ? 1.0 : 0.0;
      Y[int64_t(c) * n + r] = (e - s) / L[int64_t(r) * n + r];
    }
    __syncthreads();
  }
  for (int r = n - 1; r >= 0; --r) {
    double acc = 0.0;
    if (active)
      for (int k = r + 1 + part; k < n; k += 8) acc += L[int64_t(k) * n + r] * Y[int64_t(c) * n + k];
    red[part][c] = acc;
    __syncthreads();
    if (part == 0 && active) {
      double s = 0.0;
      for (int q = 0; q < 8; ++q) s += red[q][c];
      Y[int64_t(c) * n + r] = (Y[int64_t(c) * n + r] - s) / L[int64_t(r) * n + r];
    }
    __syncthreads();
  }
  for (int r = part; r < n; r += 8)
    if (active) Ainv[int64_t(r) * n + col] = Y[int64_t(c) * n + r];
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

gdsw_status read_err(int* d_err, cudaStream_t s, const char* what) {
  int h = 0;
  GDSW_CK(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (h & ERR_BREAKDOWN) {
    set_error("%s: non-positive or zero pivot", what);
    return GDSW_ERR_BREAKDOWN;
  }
  return GDSW_OK;
}

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, int64_t(kNumSMs) * 32)));
}

// Temporary device buffers freed when the setup returns.
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() { for (void* p : ptrs) cudaFree(p); }
  template <class T>
  gdsw_status get(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of %zu scratch bytes failed", count * sizeof(T));
      return GDSW_ERR_OUT_OF_MEMORY;
    }
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return GDSW_OK;
  }
  template <class T>
  gdsw_status put(T** p, const std::vector<T>& v, cudaStream_t s) {
    GDSW_TRY(get(p, v.size()));
    if (!v.empty())
      GDSW_CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return GDSW_OK;
  }
};

// Factor every matrix of a batch of band problems; chunks keep the band
// storage under `budget` bytes.  `fill(p0, p1, band, boff)` assembles the
// bands of problems [p0, p1) into the zeroed buffer, `after(p0, p1, band,
// boff)` consumes the factors.
template <class Fill, class After>
gdsw_status band_batches(int np, const std::vector<int>& bn, const std::vector<int>& bw,
                         size_t budget, cudaStream_t s, int* d_err, Fill fill, After after) {
  Scratch sc;
  int* d_bn = nullptr;
  int* d_bw = nullptr;
  GDSW_TRY(sc.put(&d_bn, bn, s));
  GDSW_TRY(sc.put(&d_bw, bw, s));
  std::vector<int64_t> boff(np + 1, 0);
  for (int p = 0; p < np; ++p) boff[p + 1] = boff[p] + int64_t(bn[p]) * (bw[p] + 1);
  int64_t maxone = 0;
  for (int p = 0; p < np; ++p) maxone = std::max<int64_t>(maxone, boff[p + 1] - boff[p]);
  const int64_t cap = std::max<int64_t>(maxone, static_cast<int64_t>(budget / sizeof(double)));
  double* band = nullptr;
  GDSW_TRY(sc.get(&band, static_cast<size_t>(std::min<int64_t>(cap, boff[np]))));
  int64_t* d_boff = nullptr;
  GDSW_TRY(sc.get(&d_boff, np + 1));
  int p0 = 0;
  int maxw = 0;
  for (int p = 0; p < np; ++p) maxw = std::max(maxw, bw[p]);
  while (p0 < np) {
    int p1 = p0;
    while (p1 < np && boff[p1 + 1] - boff[p0] <= cap) ++p1;
    std::vector<int64_t> loc(np + 1, 0);
    for (int p = p0; p <= p1 && p <= np; ++p) loc[p] = boff[p] - boff[p0];
    GDSW_CK(cudaMemcpyAsync(d_boff, loc.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    GDSW_CK(cudaMemsetAsync(band, 0, (boff[p1] - boff[p0]) * sizeof(double), s));
    GDSW_TRY(fill(p0, p1, band, d_boff));
    const size_t shm = std::max<size_t>(sizeof(double), size_t(maxw) * sizeof(double));
    if (shm > 200 * 1024) { set_error("band width %d too large for the banded Cholesky", maxw); return GDSW_ERR_UNSUPPORTED; }
    if (shm > 48 * 1024)
      GDSW_CK(allow_max_dynamic_smem(k_band_cholesky));
    k_band_cholesky<<<p1 - p0, 512, shm, s>>>(band, d_boff, d_bn, d_bw, p0, d_err);
    GDSW_CK(cudaGetLastError());
    GDSW_TRY(after(p0, p1, band, d_boff, d_bn, d_bw));
    GDSW_CK(cudaStreamSynchronize(s));   // the band buffer is reused by the next chunk
    p0 = p1;
  }
  return GDSW_OK;
}

}  // namespace

gdsw_status numeric_setup(Ctx* c, const Plan& P, const gdsw_csr* A, const double* Z, int nn,
                          cudaStream_t s) {
  const gdsw_options& o = c->opt;
  const bool exact = o.local_solver == GDSW_LOCAL_EXACT;
  const bool ilu = o.local_solver == GDSW_LOCAL_ILU0;
  const int nsub = P.nsub;
  const int64_t nent = P.lm_col.size();
  Scratch sc;
  int* d_err = nullptr;
  GDSW_TRY(sc.get(&d_err, 1));
  GDSW_CK(cudaMemsetAsync(d_err, 0, sizeof(int), s));

  // ---- global matrix and overlap ----
  {
    std::vector<int> rp(A->rowptr, A->rowptr + P.n + 1);
    std::vector<int> ci(A->colind, A->colind + P.nnz);
    std::vector<double> va(A->val, A->val + P.nnz);
    GDSW_TRY(upload(c, &c->rowptr, rp, s));
    GDSW_TRY(upload(c, &c->colind, ci, s));
    GDSW_TRY(upload(c, &c->val, va, s));
  }
  GDSW_TRY(upload(c, &c->om_ptr, P.om_ptr, s));
  {
    // padded by four words: the pipelined local solve copies each subdomain's
    // slice from a 16-byte aligned start in whole 16-byte units
    std::vector<int> padded(P.om_dofs);
    padded.resize(P.om_dofs.size() + 4, 0);
    GDSW_TRY(upload(c, &c->om_dofs, padded, s));
  }

  // ---- local matrices ----
  double t0 = now_s();
  int *d_lm_sub_ent, *d_lm_rowptr, *d_lm_col, *d_lm_gent, *d_lm_diag, *d_lm_tpos;
  uint16_t* d_lm_row;
  GDSW_TRY(sc.put(&d_lm_sub_ent, P.lm_sub_ent, s));
  GDSW_TRY(sc.put(&d_lm_rowptr, P.lm_rowptr, s));
  GDSW_TRY(sc.put(&d_lm_col, P.lm_col, s));
  GDSW_TRY(sc.put(&d_lm_gent, P.lm_gent, s));
  GDSW_TRY(sc.put(&d_lm_diag, P.lm_diag, s));
  GDSW_TRY(sc.put(&d_lm_row, P.lm_row, s));
  double *d_sc, *d_at, *d_araw;
  GDSW_TRY(sc.get(&d_sc, P.sum_m));
  GDSW_TRY(sc.get(&d_at, nent));
  GDSW_TRY(sc.get(&d_araw, nent));
  k_extract_local<<<nsub, 256, 0, s>>>(c->val, c->om_ptr, d_lm_sub_ent, d_lm_gent, d_lm_row,
                                       d_lm_col, d_lm_diag, d_sc, d_at, d_araw, d_err);
  GDSW_CK(cudaGetLastError());

  if (!exact) {
    GDSW_TRY(read_err(d_err, s, "local matrix diagonal"));
    GDSW_TRY(sc.put(&d_lm_tpos, P.lm_tpos, s));
    double *F0, *F1, *G;
    GDSW_TRY(sc.get(&F0, nent));
    GDSW_TRY(sc.get(&F1, nent));
    GDSW_TRY(sc.get(&G, nent));
    // subdomain row base of every entry
    std::vector<int> ebase(nent);
    for (int q = 0; q < nsub; ++q)
      for (int e = P.lm_sub_ent[q]; e < P.lm_sub_ent[q + 1]; ++e) ebase[e] = P.om_ptr[q];
    int* d_ebase;
    GDSW_TRY(sc.put(&d_ebase, ebase, s));
    const int sw = std::max(0, o.sweeps_factor);
    GDSW_CK(cudaMemcpyAsync(F0, d_at, nent * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double* Fo = F0;
    double* Fn = F1;
    const int ne = static_cast<int>(nent);
    for (int q = 0; q < sw; ++q) {
      if (ilu)
        k_ilu0_sweep<<<grid_for(nent, 256), 256, 0, s>>>(ne, d_ebase, d_lm_rowptr, d_lm_col, d_lm_row,
                                                         d_lm_diag, d_lm_tpos, d_at, Fo, Fn, d_err);
      else
        k_ic0_sweep<<<grid_for(nent, 256), 256, 0, s>>>(ne, d_ebase, d_lm_rowptr, d_lm_col, d_lm_row,
                                                        d_lm_diag, d_at, Fo, Fn, d_err);
      GDSW_CK(cudaGetLastError());
      std::swap(Fo, Fn);
    }
    GDSW_TRY(read_err(d_err, s, ilu ? "ILU(0) sweeps" : "IC(0) sweeps"));
    double* F = Fo;
    k_unscale<<<grid_for(nent, 256), 256, 0, s>>>(static_cast<int>(nent), ilu ? 1 : 0, nullptr,
                                                  d_lm_row, d_lm_col, d_ebase, d_sc, F, G);
    GDSW_CK(cudaGetLastError());
    // level-sliced ELL in the apply precision
    struct Side { const EllPlan* E; int** sub; int4** lev; uint16_t** lrows; uint16_t** col; void** val; void** dinv; };
    Side sides[2] = {{&P.L, &c->L_sub_lev, &c->L_lev, &c->L_lrows, &c->L_col, &c->L_val, &c->L_dinv},
                     {&P.U, &c->U_sub_lev, &c->U_lev, &c->U_lrows, &c->U_col, &c->U_val, &c->U_dinv}};
    for (Side& sd : sides) {
      const EllPlan& E = *sd.E;
      std::vector<int4> lev(E.lev_nr.size());
      for (size_t l = 0; l < lev.size(); ++l)
        lev[l] = make_int4(E.lev_start[l], E.lev_nr[l], E.lev_K[l], E.lev_off[l]);
      GDSW_TRY(upload(c, sd.sub, E.sub_lev, s));
      GDSW_TRY(upload(c, sd.lev, lev, s));
      GDSW_TRY(upload(c, sd.lrows, E.lrows, s));
      GDSW_TRY(upload(c, sd.col, E.col, s));
      int *d_src, *d_dsrc;
      GDSW_TRY(sc.put(&d_src, E.src, s));
      GDSW_TRY(sc.put(&d_dsrc, E.dsrc, s));
      if (c->fp32) {
        float *v, *d;
        GDSW_TRY(dalloc(c, &v, E.slots));
        GDSW_TRY(dalloc(c, &d, P.sum_m));
        k_pack_ell<float><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, G, v);
        k_pack_dinv<float><<<grid_for(P.sum_m, 256), 256, 0, s>>>(P.sum_m, d_dsrc, G, d);
        *sd.val = v; *sd.dinv = d;
      } else {
        double *v, *d;
        GDSW_TRY(dalloc(c, &v, E.slots));
        GDSW_TRY(dalloc(c, &d, P.sum_m));
        k_pack_ell<double><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, G, v);
        k_pack_dinv<double><<<grid_for(P.sum_m, 256), 256, 0, s>>>(P.sum_m, d_dsrc, G, d);
        *sd.val = v; *sd.dinv = d;
      }
      GDSW_CK(cudaGetLastError());
    }
    c->max_levels = std::max(P.L.max_levels, P.U.max_levels);
    // Per-level records for the pipelined level-scheduled solve: for every
    // subdomain its L levels then its U levels (wide levels split into pieces),
    // each record 16-byte aligned and one bulk copy:
    //   int4 {rows, stored width, values offset, columns offset} | int4 {in-node
    //   offset, layout, 0, 0} | rows x uint16 local row | rows x T inverse
    //   diagonal | width*rows x T values | width*rows x uint16 columns
    //   [| (dpn-1)*rows + 1 x T in-node coefficients]
    // every section padded to 16 bytes.  Layouts: 0 column-major; 1 row-major
    // padded to 4 (widths 1-4, one unknown per node); 2 by node (several
    // unknowns per node): the entries coupling a row to other nodes
    // column-major, those to earlier-solved rows of its own node as
    // coefficients by solve step (row t, step q at t*(dpn-1)+q; one trailing
    // zero absorbs the padding).  More than 4 unknowns per node: no records
    // (the unpipelined kernel solves).
    if (P.dpn <= 4) {
      const size_t vb = c->fp16 ? sizeof(__half) : c->fp32 ? sizeof(float) : sizeof(double);
      const size_t rcap = record_cap();
      const int Gn = P.dpn;
      auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
      struct RecLayout { int layout; size_t K, o_l, o_d, o_v, o_c, o_i, end; };
      // solve step of local column `col` inside its node (L: increasing, U: decreasing)
      auto step_of = [&](bool lower, int col) { return lower ? col % Gn : Gn - 1 - col % Gn; };
      auto layout_of = [&](const EllPlan& E, bool lower, int l, size_t t0, size_t nr) {
        RecLayout R;
        const size_t L_nr = E.lev_nr[l], K = E.lev_K[l];
        if (Gn > 1) {
          size_t koff = 0;
          for (size_t t = 0; t < nr; ++t) {
            const int row = E.lrows[E.lev_start[l] + t0 + t];
            size_t cnt = 0;
            for (size_t k = 0; k < K; ++k) {
              const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + t0 + t;
              if (E.src[slot] >= 0 && E.col[slot] / Gn != row / Gn) ++cnt;
            }
            koff = std::max(koff, cnt);
          }
          R.layout = 2;
          R.K = koff;
        } else {
          R.layout = record_width(E.lev_K[l]) == 4 ? 1 : 0;
          R.K = record_width(E.lev_K[l]);
        }
        (void)lower;
        R.o_l = 32;
        R.o_d = R.o_l + a16(2 * nr);
        R.o_v = R.o_d + a16(nr * vb);
        R.o_c = R.o_v + a16(R.K * nr * vb);
        R.o_i = R.o_c + a16(2 * R.K * nr);
        R.end = R.layout == 2 ? R.o_i + a16((size_t(Gn - 1) * nr + 1) * vb) : R.o_i;
        return R;
      };
      std::vector<int> rec_ptr(nsub + 1, 0);
      std::vector<uint32_t> rec_off16, rec_bytes;
      std::vector<int> rec_lev, rec_t0;            // level and first row of every record
      std::vector<char> rec_is_L;
      std::vector<uint32_t> valposL(P.L.slots), valposU(P.U.slots), dinvposL(P.sum_m), dinvposU(P.sum_m);
      size_t total = 0;
      for (int pass = 0; pass < 2; ++pass) {      // pass 0 sizes, pass 1 fills
        total = 0;
        for (int q = 0; q < nsub; ++q) {
          for (int side = 0; side < 2; ++side) {
            const EllPlan& E = side == 0 ? P.L : P.U;
            const bool lower = side == 0;
            for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l) {
              // a wide level becomes several records (rows are independent
              // within a level, node groups kept whole)
              const size_t L_nr = E.lev_nr[l], K = E.lev_K[l];
              const size_t piece = record_piece_rows(E.lev_nr[l], E.lev_K[l], Gn, vb, rcap);
              for (size_t t0 = 0; t0 < L_nr; t0 += piece) {
                const size_t nr = std::min(piece, L_nr - t0);
                const RecLayout R = layout_of(E, lower, l, t0, nr);
                if (pass == 1) {
                  rec_off16.push_back(static_cast<uint32_t>(total / 16));
                  rec_bytes.push_back(static_cast<uint32_t>(R.end));
                  rec_lev.push_back(l);
                  rec_t0.push_back(static_cast<int>(t0));
                  rec_is_L.push_back(lower);
                  uint32_t* dp = lower ? dinvposL.data() : dinvposU.data();
                  uint32_t* vp = lower ? valposL.data() : valposU.data();
                  for (size_t t = 0; t < nr; ++t)
                    dp[E.lev_start[l] + t0 + t] = static_cast<uint32_t>((total + R.o_d + t * vb) / vb);
                  for (size_t t = 0; t < nr; ++t) {
                    const int row = E.lrows[E.lev_start[l] + t0 + t];
                    size_t koff = 0;
                    for (size_t k = 0; k < K; ++k) {
                      const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + t0 + t;
                      size_t pos;
                      if (R.layout == 0) pos = R.o_v + (k * nr + t) * vb;
                      else if (R.layout == 1) pos = R.o_v + (t * 4 + k) * vb;
                      else if (E.src[slot] < 0) pos = R.o_i + size_t(Gn - 1) * nr * vb;     // padding: the zero
                      else if (E.col[slot] / Gn == row / Gn)
                        pos = R.o_i + (t * (Gn - 1) + step_of(lower, E.col[slot])) * vb;
                      else
                        pos = R.o_v + (koff++ * nr + t) * vb;
                      vp[slot] = static_cast<uint32_t>((total + pos) / vb);
                    }
                  }
                }
                total += R.end;
              }
            }
          }
          if (pass == 1) rec_ptr[q + 1] = static_cast<int>(rec_off16.size());
        }
        if (total / 16 >= (size_t(1) << 32) || total / vb >= (size_t(1) << 32)) {
          set_error("factor stream too large"); return GDSW_ERR_UNSUPPORTED;
        }
      }
      std::vector<uint8_t> host(total, 0);
      size_t stage = 16;
      for (size_t rr = 0; rr < rec_off16.size(); ++rr) {
        const bool lower = rec_is_L[rr];
        const EllPlan& E = lower ? P.L : P.U;
        const int l = rec_lev[rr];
        const size_t L_nr = E.lev_nr[l], K = E.lev_K[l];
        const size_t t0 = rec_t0[rr];
        const size_t nr = std::min(size_t(record_piece_rows(E.lev_nr[l], E.lev_K[l], Gn, vb, rcap)), L_nr - t0);
        const RecLayout R = layout_of(E, lower, l, t0, nr);
        const size_t base = size_t(rec_off16[rr]) * 16;
        // word 5: the layout, plus kRecUpper for the records of the U sweep and
        // kRecLevelEnd for the last record of each level
        const bool level_end = t0 + nr == L_nr;
        const int hdr[8] = {static_cast<int>(nr), static_cast<int>(R.K), static_cast<int>(R.o_v),
                            static_cast<int>(R.o_c), static_cast<int>(R.o_i),
                            R.layout | (lower ? 0 : kRecUpper) | (level_end ? kRecLevelEnd : 0),
                            static_cast<int>(R.end), 1};
        std::memcpy(&host[base], hdr, 32);
        std::memcpy(&host[base + R.o_l], &E.lrows[E.lev_start[l] + t0], 2 * nr);
        uint16_t* cc = reinterpret_cast<uint16_t*>(&host[base + R.o_c]);
        for (size_t t = 0; t < nr; ++t) {
          const int row = E.lrows[E.lev_start[l] + t0 + t];
          size_t koff = 0;
          for (size_t k = 0; k < R.K; ++k) {
            if (R.layout == 1) {
              cc[t * 4 + k] = k < K ? E.col[E.lev_off[l] + k * L_nr + t0 + t] : static_cast<uint16_t>(row);
            } else if (R.layout == 0) {
              cc[k * nr + t] = E.col[E.lev_off[l] + k * L_nr + t0 + t];
            }
          }
          if (R.layout == 2) {
            // off-node columns in entry order, then the row itself as padding
            for (size_t k = 0; k < K; ++k) {
              const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + t0 + t;
              if (E.src[slot] >= 0 && E.col[slot] / Gn != row / Gn) cc[koff++ * nr + t] = E.col[slot];
            }
            for (; koff < R.K; ++koff) cc[koff * nr + t] = static_cast<uint16_t>(row);
          }
        }
        stage = std::max<size_t>(stage, rec_bytes[rr]);
      }
      // Consecutive records of a subdomain are contiguous in the stream: pack
      // them greedily into one bulk copy while the pack stays within a ring
      // stage: the largest single record, or GDSW_PACK_BYTES if larger (fewer,
      // larger copies).  The first record of a pack carries the pack's record
      // count (header word 7); every record its own size (word 6), so the
      // consumers step through the pack.
      if (const char* e = getenv("GDSW_PACK_BYTES")) {
        const long want = atol(e);
        if (want > 0) stage = std::max<size_t>(stage, (static_cast<size_t>(want) + 15) & ~size_t(15));
      }
      std::vector<int> pk_ptr(nsub + 1, 0);
      std::vector<uint32_t> pk_off16, pk_bytes;
      for (int q = 0; q < nsub; ++q) {
        for (int rr = rec_ptr[q]; rr < rec_ptr[q + 1];) {
          size_t bytes = rec_bytes[rr];
          int cnt = 1;
          while (rr + cnt < rec_ptr[q + 1] && bytes + rec_bytes[rr + cnt] <= stage) bytes += rec_bytes[rr + cnt++];
          int* first = reinterpret_cast<int*>(&host[size_t(rec_off16[rr]) * 16]);
          first[7] = cnt;
          pk_off16.push_back(rec_off16[rr]);
          pk_bytes.push_back(static_cast<uint32_t>(bytes));
          rr += cnt;
        }
        pk_ptr[q + 1] = static_cast<int>(pk_off16.size());
      }
      uint8_t* d_stream;
      GDSW_TRY(upload(c, &d_stream, host, s));
      c->rec_stream = d_stream;
      GDSW_TRY(upload(c, &c->rec_ptr, pk_ptr, s));
      GDSW_TRY(upload(c, &c->rec_off16, pk_off16, s));
      GDSW_TRY(upload(c, &c->rec_bytes, pk_bytes, s));
      c->rec_stage_bytes = static_cast<int>(stage);
      int maxK = 0;
      for (int kk : P.L.lev_K) maxK = std::max(maxK, kk);
      for (int kk : P.U.lev_K) maxK = std::max(maxK, kk);
      c->rec_max_width = maxK;
      int maxR = 0;
      for (int nr : P.L.lev_nr) maxR = std::max(maxR, nr);
      for (int nr : P.U.lev_nr) maxR = std::max(maxR, nr);
      c->rec_max_rows = maxR;
      c->rec_total_bytes = static_cast<int64_t>(total);
      for (int side = 0; side < 2; ++side) {
        const EllPlan& E = side == 0 ? P.L : P.U;
        uint32_t *d_vp, *d_dp;
        int *d_src, *d_dsrc;
        GDSW_TRY(sc.put(&d_vp, side == 0 ? valposL : valposU, s));
        GDSW_TRY(sc.put(&d_dp, side == 0 ? dinvposL : dinvposU, s));
        GDSW_TRY(sc.put(&d_src, E.src, s));
        GDSW_TRY(sc.put(&d_dsrc, E.dsrc, s));
        if (c->fp16)
          k_fill_records<__half><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                       reinterpret_cast<__half*>(d_stream));
        else if (c->fp32)
          k_fill_records<float><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                      reinterpret_cast<float*>(d_stream));
        else
          k_fill_records<double><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                       reinterpret_cast<double*>(d_stream));
        GDSW_CK(cudaGetLastError());
      }
    }
    // Row programs for the level-scheduled solve (k_local_steps): one unknown
    // per node, FP32, at most three off-diagonal entries per row (IC(0)/ILU(0)
    // of 7-point stencils).  Every row of every
    // level becomes one 24-byte instruction in two arrays, A: float4 {a0, a1,
    // a2, inverse diagonal} and C: uint2 {c0 | c1 << 16, c2 | row << 16} (the
    // level-sliced ELL's entries in slot order, rows narrower than three padded
    // with a zero entry on the row itself, as the row-major records are).  A
    // subdomain's program is its L levels then its U levels, each level cut
    // into steps of at most kStepRows rows (thread t takes row t of a step); a
    // step is int2 {first instruction, rows | 1 << 16 when the level ends}.
    if (P.dpn == 1 && c->fp32 && !c->fp16 && o.trsv == GDSW_TRSV_LEVELSCHED && c->rec_max_width <= 3 &&
        P.sum_m > 0) {
      std::vector<int> sp(nsub + 1, 0);
      std::vector<int2> steps;
      std::vector<uint32_t> ccode;               // two words per instruction
      std::vector<uint32_t> vposL(P.L.slots), vposU(P.U.slots), dposL(P.sum_m), dposU(P.sum_m);
      int64_t ninstr = 0;
      int max_steps = 0;
      for (int q = 0; q < nsub; ++q) {
        for (int side = 0; side < 2; ++side) {
          const EllPlan& E = side == 0 ? P.L : P.U;
          uint32_t* vp = side == 0 ? vposL.data() : vposU.data();
          uint32_t* dp = side == 0 ? dposL.data() : dposU.data();
          for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l) {
            const int L_nr = E.lev_nr[l], K = E.lev_K[l];
            for (int t0 = 0; t0 < L_nr; t0 += kStepRows) {
              const int nr = std::min(kStepRows, L_nr - t0);
              steps.push_back(make_int2(static_cast<int>(ninstr), nr | (t0 + nr == L_nr ? 1 << 16 : 0)));
              for (int t = t0; t < t0 + nr; ++t) {
                const int row = E.lrows[E.lev_start[l] + t];
                uint16_t cc[3];
                for (int k = 0; k < 3; ++k) {
                  if (k < K) {
                    const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + t;
                    cc[k] = E.col[slot];
                    vp[slot] = static_cast<uint32_t>(ninstr * 4 + k);
                  } else {
                    cc[k] = static_cast<uint16_t>(row);
                  }
                }
                dp[E.lev_start[l] + t] = static_cast<uint32_t>(ninstr * 4 + 3);
                ccode.push_back(uint32_t(cc[0]) | uint32_t(cc[1]) << 16);
                ccode.push_back(uint32_t(cc[2]) | uint32_t(row) << 16);
                ++ninstr;
              }
            }
          }
        }
        sp[q + 1] = static_cast<int>(steps.size());
        max_steps = std::max(max_steps, sp[q + 1] - sp[q]);
      }
      if (ninstr * 4 >= (int64_t(1) << 32)) { set_error("row programs too large"); return GDSW_ERR_UNSUPPORTED; }
      float* d_a;
      GDSW_TRY(dalloc(c, &d_a, size_t(ninstr) * 4));
      GDSW_CK(cudaMemsetAsync(d_a, 0, sizeof(float) * size_t(ninstr) * 4, s));
      uint32_t* d_c;
      GDSW_TRY(upload(c, &d_c, ccode, s));
      int2* d_steps;
      GDSW_TRY(upload(c, &d_steps, steps, s));
      GDSW_TRY(upload(c, &c->step_ptr, sp, s));
      c->step_a = d_a;
      c->step_c = d_c;
      c->steps = d_steps;
      c->step_max = max_steps;
      for (int side = 0; side < 2; ++side) {
        const EllPlan& E = side == 0 ? P.L : P.U;
        uint32_t *d_vp, *d_dp;
        int *d_src, *d_dsrc;
        GDSW_TRY(sc.put(&d_vp, side == 0 ? vposL : vposU, s));
        GDSW_TRY(sc.put(&d_dp, side == 0 ? dposL : dposU, s));
        GDSW_TRY(sc.put(&d_src, E.src, s));
        GDSW_TRY(sc.put(&d_dsrc, E.dsrc, s));
        k_fill_records<float><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                    d_a);
        GDSW_CK(cudaGetLastError());
      }
    }
    // Node programs for the level-scheduled solve with three unknowns per node
    // (k_local_nodes; FP32): the rows of a node share their couplings to other
    // nodes, so per subdomain, sweep (L then U) and level, pieces of at most
    // kNodePieceBytes hold for each node: its index, its three inverse
    // diagonals and in-node coefficients by solve step (float[8]: d0, d1, d2,
    // c10, c20, c21), the union of its rows' off-node columns (uint16, K per
    // node: the level's widest, rounded up to a multiple of 8, padded with the
    // node's first row) and the three rows' values over that union
    // (float[3][K], zero where a row lacks the column or on padding).  Section layout: int4
    // {nodes | U sweep << 16, K, columns offset, values offset} | uint16 node[N] | float[N][8] |
    // uint16[N][K] | float[N][3][K], each 16-byte aligned.  Values are placed
    // on the device (k_fill_records) from the factor; ELL padding goes to a
    // spare element at the end.
    if (P.dpn == 3 && c->fp32 && !c->fp16 && o.trsv == GDSW_TRSV_LEVELSCHED && P.sum_m > 0) {
      auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
      std::vector<NodePiece> pieces;
      std::vector<int> pptr;
      size_t total = 0, maxb = 0;
      const bool ok = plan_node_pieces(P, node_piece_cap(), &pieces, &pptr, &total, &maxb);
      if (ok) {
        const size_t dummy = total / 4;            // float element absorbing ELL padding
        std::vector<uint8_t> host(total + 16, 0);
        std::vector<uint32_t> vpos[2] = {std::vector<uint32_t>(P.L.slots, uint32_t(dummy)),
                                         std::vector<uint32_t>(P.U.slots, uint32_t(dummy))};
        std::vector<uint32_t> dpos[2] = {std::vector<uint32_t>(P.sum_m, uint32_t(dummy)),
                                         std::vector<uint32_t>(P.sum_m, uint32_t(dummy))};
        std::vector<int4> ptab(pieces.size());
        for (size_t pi = 0; pi < pieces.size(); ++pi) {
          const NodePiece& pc = pieces[pi];
          const EllPlan& E = pc.side == 0 ? P.L : P.U;
          const int l = pc.lev, L_nr = E.lev_nr[l], N = pc.nodes, K = pc.K;
          const size_t o_node = 16, o_coef = o_node + a16(2 * size_t(N)), o_col = o_coef + 32 * size_t(N),
                       o_val = o_col + a16(2 * size_t(N) * K);
          const int hdr[4] = {N | (pc.side << 16), K, static_cast<int>(o_col), static_cast<int>(o_val)};
          std::memcpy(&host[pc.off], hdr, 16);
          uint16_t* nodes = reinterpret_cast<uint16_t*>(&host[pc.off + o_node]);
          uint16_t* cols = reinterpret_cast<uint16_t*>(&host[pc.off + o_col]);
          for (int gi = 0; gi < N; ++gi) {
            const int tbase = 3 * (pc.t0 + gi);
            const int row0 = E.lrows[E.lev_start[l] + tbase];
            const int g = row0 / 3;
            nodes[gi] = static_cast<uint16_t>(g);
            std::vector<uint16_t> u;
            for (int st = 0; st < 3; ++st)
              for (int k = 0; k < E.lev_K[l]; ++k) {
                const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + tbase + st;
                if (E.src[slot] >= 0 && E.col[slot] / 3 != g) u.push_back(E.col[slot]);
              }
            std::sort(u.begin(), u.end());
            u.erase(std::unique(u.begin(), u.end()), u.end());
            for (int k = 0; k < K; ++k)
              cols[size_t(gi) * K + k] = k < static_cast<int>(u.size()) ? u[k] : static_cast<uint16_t>(row0);
            for (int st = 0; st < 3; ++st) {
              const int t = tbase + st;
              dpos[pc.side][E.lev_start[l] + t] = static_cast<uint32_t>((pc.off + o_coef + 32 * size_t(gi)) / 4 + st);
              for (int k = 0; k < E.lev_K[l]; ++k) {
                const int64_t slot = E.lev_off[l] + int64_t(k) * L_nr + t;
                if (E.src[slot] < 0) continue;
                const int col = E.col[slot];
                size_t fpos;
                if (col / 3 == g) {
                  // in-node coefficient of step st on the step that solved col
                  const int sp = pc.side == 0 ? col % 3 : 2 - col % 3;
                  const int ci = st == 1 ? 0 : (sp == 0 ? 1 : 2);      // c10, c20, c21
                  fpos = (pc.off + o_coef + 32 * size_t(gi)) / 4 + 3 + ci;
                } else {
                  const int k2 = static_cast<int>(std::lower_bound(u.begin(), u.end(), static_cast<uint16_t>(col)) - u.begin());
                  fpos = (pc.off + o_val) / 4 + (size_t(gi) * 3 + st) * K + k2;
                }
                vpos[pc.side][slot] = static_cast<uint32_t>(fpos);
              }
            }
          }
          ptab[pi] = make_int4(static_cast<int>(pc.off / 16), static_cast<int>(pc.bytes), 0, 0);
        }
        uint8_t* d_stream;
        GDSW_TRY(upload(c, &d_stream, host, s));
        GDSW_TRY(upload(c, &c->node_ptr, pptr, s));
        GDSW_TRY(upload(c, &c->node_piece, ptab, s));
        c->node_stream = d_stream;
        c->node_slot_bytes = static_cast<int>(maxb);
        for (int side = 0; side < 2; ++side) {
          const EllPlan& E = side == 0 ? P.L : P.U;
          uint32_t *d_vp, *d_dp;
          int *d_src, *d_dsrc;
          GDSW_TRY(sc.put(&d_vp, vpos[side], s));
          GDSW_TRY(sc.put(&d_dp, dpos[side], s));
          GDSW_TRY(sc.put(&d_src, E.src, s));
          GDSW_TRY(sc.put(&d_dsrc, E.dsrc, s));
          k_fill_records<float><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                      reinterpret_cast<float*>(d_stream));
          GDSW_CK(cudaGetLastError());
        }
      }
    }
    // Resident blocks for the Jacobi sweeps (Sec. V-B3): per subdomain and
    // triangle one block that a CTA copies into shared memory once and sweeps
    // there: int4 {rows m, width K, values offset, columns offset} | m x T
    // inverse diagonal | K*m x T values | K*m x uint16 columns, slot k of local
    // row i at k*m + i, every section 16-byte aligned.  A row's entries keep
    // the order of the level-sliced ELL (so each sum is formed as by the
    // unpipelined Jacobi kernel); rows shorter than K are padded with a zero
    // entry pointing at the row itself.  Blocks are in subdomain order, L then
    // U; one spare 16 bytes at the end absorb the ELL's own padding entries.
    if (o.trsv == GDSW_TRSV_JACOBI) {
      const size_t vb = c->fp16 ? sizeof(__half) : c->fp32 ? sizeof(float) : sizeof(double);
      auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
      std::vector<uint32_t> joff(size_t(2) * nsub), jbytes(size_t(2) * nsub);
      std::vector<int> jK(size_t(2) * nsub, 0);
      size_t total = 0, maxb[2] = {0, 0};
      for (int q = 0; q < nsub; ++q) {
        const size_t m = size_t(P.om_ptr[q + 1] - P.om_ptr[q]);
        for (int side = 0; side < 2; ++side) {
          const EllPlan& E = side == 0 ? P.L : P.U;
          int K = 0;
          for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l)
            for (int t = 0; t < E.lev_nr[l]; ++t) {
              int w = 0;
              for (int k = 0; k < E.lev_K[l]; ++k) w += E.src[E.lev_off[l] + int64_t(k) * E.lev_nr[l] + t] >= 0;
              K = std::max(K, w);
            }
          jK[2 * q + side] = K;
          const size_t bytes = 16 + a16(m * vb) + a16(size_t(K) * m * vb) + a16(size_t(K) * m * 2);
          joff[2 * q + side] = static_cast<uint32_t>(total / 16);
          jbytes[2 * q + side] = static_cast<uint32_t>(bytes);
          maxb[side] = std::max(maxb[side], bytes);
          total += bytes;
          if (total / 16 >= (size_t(1) << 32) || total / vb >= (size_t(1) << 32)) {
            set_error("Jacobi blocks too large"); return GDSW_ERR_UNSUPPORTED;
          }
        }
      }
      const size_t dummy = total / vb;            // element receiving the ELL padding
      std::vector<uint8_t> host(total + 16, 0);
      std::vector<uint32_t> vpos[2] = {std::vector<uint32_t>(P.L.slots), std::vector<uint32_t>(P.U.slots)};
      std::vector<uint32_t> dpos[2] = {std::vector<uint32_t>(P.sum_m), std::vector<uint32_t>(P.sum_m)};
      for (int q = 0; q < nsub; ++q) {
        const int m = P.om_ptr[q + 1] - P.om_ptr[q];
        for (int side = 0; side < 2; ++side) {
          const EllPlan& E = side == 0 ? P.L : P.U;
          const int K = jK[2 * q + side];
          const size_t base = size_t(joff[2 * q + side]) * 16;
          const size_t o_d = 16, o_v = o_d + a16(size_t(m) * vb), o_c = o_v + a16(size_t(K) * m * vb);
          const int hdr[4] = {m, K, static_cast<int>(o_v), static_cast<int>(o_c)};
          std::memcpy(&host[base], hdr, 16);
          uint16_t* cc = reinterpret_cast<uint16_t*>(&host[base + o_c]);
          for (int i = 0; i < m; ++i)
            for (int k = 0; k < K; ++k) cc[size_t(k) * m + i] = static_cast<uint16_t>(i);
          for (int l = E.sub_lev[q]; l < E.sub_lev[q + 1]; ++l) {
            const int nr = E.lev_nr[l];
            for (int t = 0; t < nr; ++t) {
              const int row = E.lrows[E.lev_start[l] + t];
              dpos[side][E.lev_start[l] + t] = static_cast<uint32_t>((base + o_d) / vb + row);
              int kk = 0;
              for (int k = 0; k < E.lev_K[l]; ++k) {
                const int64_t slot = E.lev_off[l] + int64_t(k) * nr + t;
                if (E.src[slot] >= 0) {
                  cc[size_t(kk) * m + row] = E.col[slot];
                  vpos[side][slot] = static_cast<uint32_t>((base + o_v) / vb + size_t(kk) * m + row);
                  ++kk;
                } else {
                  vpos[side][slot] = static_cast<uint32_t>(dummy);
                }
              }
            }
          }
        }
      }
      uint8_t* d_js;
      GDSW_TRY(upload(c, &d_js, host, s));
      c->jac_stream = d_js;
      GDSW_TRY(upload(c, &c->jac_off16, joff, s));
      GDSW_TRY(upload(c, &c->jac_bytes, jbytes, s));
      c->jac_max_bytes[0] = static_cast<int>(maxb[0]);
      c->jac_max_bytes[1] = static_cast<int>(maxb[1]);
      for (int side = 0; side < 2; ++side) {
        const EllPlan& E = side == 0 ? P.L : P.U;
        uint32_t *d_vp, *d_dp;
        int *d_src, *d_dsrc;
        GDSW_TRY(sc.put(&d_vp, vpos[side], s));
        GDSW_TRY(sc.put(&d_dp, dpos[side], s));
        GDSW_TRY(sc.put(&d_src, E.src, s));
        GDSW_TRY(sc.put(&d_dsrc, E.dsrc, s));
        if (c->fp16)
          k_fill_records<__half><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                       reinterpret_cast<__half*>(d_js));
        else if (c->fp32)
          k_fill_records<float><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                      reinterpret_cast<float*>(d_js));
        else
          k_fill_records<double><<<grid_for(E.slots, 256), 256, 0, s>>>(E.slots, d_src, d_vp, P.sum_m, d_dsrc, d_dp, G,
                                                                       reinterpret_cast<double*>(d_js));
        GDSW_CK(cudaGetLastError());
      }
    }
    GDSW_CK(cudaStreamSynchronize(s));   // scratch of this stage is released below
  }
  c->stats.setup_phase_seconds[1] = now_s() - t0;

  // ---- Phi_Gamma: MGS per coarse-space owner over its weighted support ----
  // (GDSW: every interface component owns itself with weight 1; rGDSW: the
  // vertices own the edges and faces of their closure with weight 1/N_c.)
  t0 = now_s();
  std::vector<int> comp_rank(P.ncomp, 0);
  double* d_Q = nullptr;
  int zcols = nn;
  const bool coarse = (o.coarse == GDSW_COARSE_GDSW || o.coarse == GDSW_COARSE_RGDSW) && P.ncomp > 0;
  SupportPlan S;
  GDSW_TRY(build_supports(P, &S));
  const int nown = static_cast<int>(S.owners.size());
  int *d_supp_ptr = nullptr, *d_supp_dof = nullptr, *d_supp_comp = nullptr, *d_supp_row = nullptr;
  if (coarse && nown > 0) {
    double* d_Z;
    std::vector<double> zh;
    if (Z == nullptr || nn == 0) { zh.assign(P.n, 1.0); zcols = 1; }
    else zh.assign(Z, Z + int64_t(P.n) * nn);
    GDSW_TRY(sc.put(&d_Z, zh, s));
    double* d_supp_w;
    GDSW_TRY(sc.put(&d_supp_ptr, S.supp_ptr, s));
    GDSW_TRY(sc.put(&d_supp_dof, S.supp_dof, s));
    GDSW_TRY(sc.put(&d_supp_comp, S.supp_comp, s));
    GDSW_TRY(sc.put(&d_supp_row, S.supp_row, s));
    GDSW_TRY(sc.put(&d_supp_w, S.supp_w, s));
    GDSW_TRY(sc.get(&d_Q, size_t(S.supp_ptr[nown]) * zcols));
    int* d_rank;
    GDSW_TRY(sc.get(&d_rank, nown));
    k_mgs<<<nown, 128, 0, s>>>(d_supp_ptr, d_supp_dof, d_supp_w, d_Z, P.n, zcols, d_Q, d_rank);
    GDSW_CK(cudaGetLastError());
    std::vector<int> orank(nown);
    GDSW_CK(cudaMemcpyAsync(orank.data(), d_rank, nown * sizeof(int), cudaMemcpyDeviceToHost, s));
    GDSW_CK(cudaStreamSynchronize(s));
    for (int q = 0; q < nown; ++q) comp_rank[S.owners[q]] = orank[q];
  }
  CoarsePlan C;
  GDSW_TRY(build_coarse_plan(P, S, comp_rank, coarse && nown > 0, &C));
  // per owner: first coarse column and column count
  std::vector<int> owner_c0(std::max(nown, 1), 0), owner_k(std::max(nown, 1), 0);
  for (int q = 0; q < nown; ++q) {
    owner_c0[q] = C.comp_c0[S.owners[q]];
    owner_k[q] = C.comp_k[S.owners[q]];
  }
  c->n0 = C.n0;
  c->nblk = C.nblk;
  GDSW_TRY(upload(c, &c->brow_ptr, C.brow_ptr, s));
  GDSW_TRY(upload(c, &c->brow_dof, C.brow_dof, s));
  GDSW_TRY(upload(c, &c->bcol_ptr, C.bcol_ptr, s));
  GDSW_TRY(upload(c, &c->bcol, C.bcol, s));
  c->n_bslots = static_cast<int>(C.bcol.size());
  if (c->fp32) {
    float* yb;
    GDSW_TRY(dalloc(c, &yb, std::max<size_t>(1, C.bcol.size())));
    c->yslot = yb;
  } else {
    double* yb;
    GDSW_TRY(dalloc(c, &yb, std::max<size_t>(1, C.bcol.size())));
    c->yslot = yb;
  }
  GDSW_TRY(upload(c, &c->phi_off, C.phi_off, s));
  GDSW_TRY(upload(c, &c->cs_ptr, C.cs_ptr, s));
  GDSW_TRY(upload(c, &c->cs_idx, C.cs_idx, s));
  GDSW_TRY(upload(c, &c->pull_ptr, C.pull_ptr, s));
  GDSW_TRY(upload(c, &c->pull_pos, C.pull_pos, s));
  GDSW_TRY(upload(c, &c->pos_blk, C.pos_blk, s));
  GDSW_TRY(upload(c, &c->chunk_blk, C.chunk_blk, s));
  GDSW_TRY(upload(c, &c->chunk_r0, C.chunk_r0, s));
  GDSW_TRY(upload(c, &c->chunk_r1, C.chunk_r1, s));
  GDSW_TRY(upload(c, &c->chunk_slot, C.chunk_slot, s));
  c->n_chunks = static_cast<int>(C.chunk_blk.size());
  c->n_cta_chunks = C.n_cta_chunks;
  // Phi^T r by eight columns at a time over each chunk's rows where the CTA
  // chunks' blocks are wide (48 columns or more on average: rigid-body coarse
  // spaces of elasticity), else by a warp per column (a fixed rule, so the
  // rounding never depends on a timing); GDSW_PHIT=wide or cols forces one
  {
    int64_t kc_sum = 0;
    for (int q = 0; q < C.n_cta_chunks; ++q)
      kc_sum += C.bcol_ptr[C.chunk_blk[q] + 1] - C.bcol_ptr[C.chunk_blk[q]];
    c->phiT_wide = C.n_cta_chunks > 0 && kc_sum >= int64_t(48) * C.n_cta_chunks;
    if (const char* e = getenv("GDSW_PHIT")) c->phiT_wide = e[0] == 'w';
  }
  c->n_slots = C.n_slots;
  c->stats.nnz_phi = C.phi_len;
  c->max_bcols = 0;
  for (int b = 0; b < C.nblk; ++b) c->max_bcols = std::max(c->max_bcols, C.bcol_ptr[b + 1] - C.bcol_ptr[b]);
  GDSW_TRY(dalloc(c, &c->partial, std::max(1, c->n_slots)));
  GDSW_TRY(dalloc(c, &c->cvec, std::max(1, C.n0)));
  GDSW_TRY(dalloc(c, &c->yvec, std::max(1, C.n0)));
  if (c->fp32) GDSW_TRY(dalloc(c, &c->yvec32, std::max(1, C.n0)));
  double* phi64 = nullptr;
  if (C.n0 > 0) {
    GDSW_TRY(sc.get(&phi64, C.phi_len));
    GDSW_CK(cudaMemsetAsync(phi64, 0, C.phi_len * sizeof(double), s));
    int *d_colpos, *d_owner_k;
    GDSW_TRY(sc.put(&d_colpos, C.supp_colpos, s));
    GDSW_TRY(sc.put(&d_owner_k, owner_k, s));
    k_copy_phig<<<nown, 256, 0, s>>>(nsub, d_supp_ptr, d_supp_comp, d_supp_row, d_colpos, d_owner_k, zcols, d_Q,
                                     c->brow_ptr, c->phi_off, phi64);
    GDSW_CK(cudaGetLastError());
  }
  c->stats.setup_phase_seconds[2] = now_s() - t0;

  // ---- Phi_I = -A_II^-1 A_IGamma Phi_Gamma (Eq. 2), banded Cholesky per interior ----
  t0 = now_s();
  if (C.n0 > 0) {
    int *d_int_ptr, *d_int_dofs, *d_dof_comp, *d_dof_comprow, *d_dof_introw;
    GDSW_TRY(sc.put(&d_int_ptr, P.int_ptr, s));
    GDSW_TRY(sc.put(&d_int_dofs, P.int_dofs, s));
    GDSW_TRY(sc.put(&d_dof_comp, P.dof_comp, s));
    GDSW_TRY(sc.put(&d_dof_comprow, P.dof_comprow, s));
    GDSW_TRY(sc.put(&d_dof_introw, P.dof_introw, s));
    std::vector<int> bn(nsub), bwv(nsub), rk(nsub);
    std::vector<int64_t> roff(nsub);
    for (int q = 0; q < nsub; ++q) {
      bn[q] = P.int_ptr[q + 1] - P.int_ptr[q];
      bwv[q] = P.int_bw[q];
      rk[q] = C.bcol_ptr[q + 1] - C.bcol_ptr[q];
      roff[q] = C.phi_off[q];
    }
    int* d_rk;
    int64_t* d_roff;
    GDSW_TRY(sc.put(&d_rk, rk, s));
    GDSW_TRY(sc.put(&d_roff, roff, s));
    int* d_bw_full;
    GDSW_TRY(sc.put(&d_bw_full, bwv, s));
    auto fill = [&](int p0, int p1, double* band, int64_t* d_boff) -> gdsw_status {
      k_assemble_interior<<<p1 - p0, 256, 0, s>>>(
          p0, c->rowptr, c->colind, c->val, d_int_ptr, d_int_dofs, d_dof_comp, d_dof_comprow,
          d_dof_introw, nsub, c->brow_ptr, c->bcol_ptr, c->bcol, c->phi_off, phi64,
          band, d_boff, d_bw_full);
      GDSW_CK(cudaGetLastError());
      return GDSW_OK;
    };
    auto after = [&](int p0, int p1, double* band, int64_t* d_boff, int* d_bn, int* d_bw) -> gdsw_status {
      k_band_solve<<<p1 - p0, 256, 0, s>>>(band, d_boff, d_bn, d_bw, phi64, d_roff, d_rk, p0);
      GDSW_CK(cudaGetLastError());
      return GDSW_OK;
    };
    GDSW_TRY(band_batches(nsub, bn, bwv, size_t(6) << 30, s, d_err, fill, after));
    GDSW_TRY(read_err(d_err, s, "interior Cholesky"));
  }
  c->stats.setup_phase_seconds[3] = now_s() - t0;

  // ---- A0 = Phi^T A Phi (one dense block per problem) and its inverse ----
  t0 = now_s();
  if (C.n0 > 0) {
    const int n0 = C.n0;
    const int np_ = P.nprob;
    std::vector<int> coarse_owner(n0), coarse_prob(n0);
    for (int q = 0; q < nown; ++q)
      for (int t = 0; t < owner_k[q]; ++t) {
        coarse_owner[owner_c0[q] + t] = q;
        coarse_prob[owner_c0[q] + t] = P.comp_prob[S.owners[q]];
      }
    std::vector<int64_t> a0_off(np_ + 1, 0);
    int maxb = 0;
    for (int q = 0; q < np_; ++q) {
      const int64_t nb = C.prob_c0[q + 1] - C.prob_c0[q];
      a0_off[q + 1] = a0_off[q] + nb * nb;
      maxb = std::max<int>(maxb, static_cast<int>(nb));
    }
    int *d_cc, *d_c0b, *d_dof_blk, *d_dof_blkrow, *d_colpos2;
    GDSW_TRY(sc.put(&d_cc, coarse_owner, s));
    GDSW_TRY(sc.put(&d_c0b, owner_c0, s));
    GDSW_TRY(sc.put(&d_colpos2, C.supp_colpos, s));
    GDSW_TRY(sc.put(&d_dof_blk, C.dof_blk, s));
    GDSW_TRY(sc.put(&d_dof_blkrow, C.dof_blkrow, s));
    GDSW_TRY(upload(c, &c->coarse_prob, coarse_prob, s));
    GDSW_TRY(upload(c, &c->prob_c0, C.prob_c0, s));
    GDSW_TRY(upload(c, &c->a0_off, a0_off, s));
    c->coarse_max_block = maxb;
    double* d_A0;
    GDSW_TRY(sc.get(&d_A0, a0_off[np_]));
    const size_t shm = size_t(maxb) * sizeof(double);
    if (shm > 227 * 1024) { set_error("coarse dimension %d too large for the A0 kernel", maxb); return GDSW_ERR_UNSUPPORTED; }
    if (shm > 48 * 1024)
      GDSW_CK(allow_max_dynamic_smem(k_coarse_rows));
    k_coarse_rows<<<n0, 32, std::max<size_t>(shm, 8), s>>>(nsub, d_cc, d_c0b, c->coarse_prob, c->prob_c0,
                                                          c->a0_off, c->rowptr, c->colind, c->val,
                                                          c->brow_ptr, d_supp_ptr, d_supp_dof, d_supp_comp,
                                                          d_supp_row, d_colpos2, c->bcol_ptr, c->bcol,
                                                          c->phi_off, phi64, d_dof_blk, d_dof_blkrow, d_A0);
    GDSW_CK(cudaGetLastError());
    c->stats.setup_phase_seconds[4] = now_s() - t0;
    t0 = now_s();
    // the inverse is formed in FP64; an FP32/FP16 apply keeps it rounded once to
    // FP32 (the whole preconditioner in single precision, Sec. VIII)
    double* a0inv64 = nullptr;
    if (c->fp32) {
      GDSW_TRY(sc.get(&a0inv64, a0_off[np_]));
      GDSW_TRY(dalloc(c, &c->A0inv32, a0_off[np_]));
      GDSW_TRY(dalloc(c, &c->cvec32, std::max(1, C.n0)));
    } else {
      GDSW_TRY(dalloc(c, &c->A0inv, a0_off[np_]));
      a0inv64 = c->A0inv;
    }
    c->stats.a0_entries = a0_off[np_];
    double* d_W;
    const int maxnbk = (maxb + NB - 1) / NB;
    GDSW_TRY(sc.get(&d_W, size_t(maxnbk) * NB * maxb));
    for (int q = 0; q < np_; ++q) {
      const int nb0 = C.prob_c0[q + 1] - C.prob_c0[q];
      if (nb0 == 0) continue;
      double* Aq = d_A0 + a0_off[q];
      const int nbk = (nb0 + NB - 1) / NB;
      for (int J = 0; J < nbk; ++J) {
        k_potrf_diag<<<1, 256, 0, s>>>(Aq, nb0, J, d_err);
        const int rest = nbk - J - 1;
        if (rest > 0) {
          k_trsm_panel<<<rest, 32, 0, s>>>(Aq, nb0, J);
          k_syrk_update<<<dim3(rest, rest), 256, 0, s>>>(Aq, nb0, J);
        }
      }
      k_chol_inverse<<<nbk, 256, 0, s>>>(Aq, nb0, d_W, a0inv64 + a0_off[q]);
    }
    if (c->fp32)
      k_convert<float><<<grid_for(a0_off[np_], 256), 256, 0, s>>>(a0_off[np_], a0inv64, c->A0inv32);
    GDSW_CK(cudaGetLastError());
    GDSW_TRY(read_err(d_err, s, "coarse Cholesky"));
    // Phi in the apply precision
    if (c->fp32) {
      float* pf;
      GDSW_TRY(dalloc(c, &pf, C.phi_len));
      k_convert<float><<<grid_for(C.phi_len, 256), 256, 0, s>>>(C.phi_len, phi64, pf);
      c->phi = pf;
    } else {
      double* pd;
      GDSW_TRY(dalloc(c, &pd, C.phi_len));
      GDSW_CK(cudaMemcpyAsync(pd, phi64, C.phi_len * sizeof(double), cudaMemcpyDeviceToDevice, s));
      c->phi = pd;
    }
    GDSW_CK(cudaGetLastError());
    GDSW_CK(cudaStreamSynchronize(s));
    c->stats.setup_phase_seconds[5] = now_s() - t0;
  }

  // ---- exact local solver: dense inverse of each A_s, or the multifrontal
  // factor when a subdomain is larger than exact_dense_max() or the inverses
  // would hold more than 2^31 entries ----
  t0 = now_s();
  if (exact) {
    GDSW_TRY(read_err(d_err, s, "local matrix"));
    std::vector<int> mn(nsub);
    std::vector<int64_t> xoff(nsub + 1, 0);
    for (int q = 0; q < nsub; ++q) {
      mn[q] = P.om_ptr[q + 1] - P.om_ptr[q];
      xoff[q + 1] = xoff[q] + int64_t(mn[q]) * mn[q];
    }
    const int64_t total = xoff[nsub];
    if (P.max_m > exact_dense_max() || total > (int64_t(1) << 31)) {
      GDSW_TRY(mf_numeric_setup(c, P, d_araw, s));
      c->stats.setup_phase_seconds[6] = now_s() - t0;
      return GDSW_OK;
    }
    double* X;
    GDSW_TRY(sc.get(&X, total));
    GDSW_CK(cudaMemsetAsync(X, 0, total * sizeof(double), s));
    int64_t* d_xoff;
    int* d_mn;
    GDSW_TRY(sc.put(&d_xoff, xoff, s));
    GDSW_TRY(sc.put(&d_mn, mn, s));
    GDSW_TRY(upload(c, &c->ainv_off, xoff, s));
    k_set_identity<<<nsub, 256, 0, s>>>(X, d_xoff, d_mn, 0);
    GDSW_CK(cudaGetLastError());
    std::vector<int> obw(P.om_bw.begin(), P.om_bw.end());
    int* d_obw;
    GDSW_TRY(sc.put(&d_obw, obw, s));
    auto fill = [&](int p0, int p1, double* band, int64_t* d_boff) -> gdsw_status {
      k_assemble_local_band<<<p1 - p0, 256, 0, s>>>(c->om_ptr, d_lm_sub_ent, d_lm_row, d_lm_col, d_araw,
                                                    band, d_boff, d_obw, p0);
      GDSW_CK(cudaGetLastError());
      return GDSW_OK;
    };
    auto after = [&](int p0, int p1, double* band, int64_t* d_boff, int* d_bn, int* d_bw) -> gdsw_status {
      k_band_solve<<<p1 - p0, 256, 0, s>>>(band, d_boff, d_bn, d_bw, X, d_xoff, d_mn, p0);
      GDSW_CK(cudaGetLastError());
      return GDSW_OK;
    };
    GDSW_TRY(band_batches(nsub, mn, obw, size_t(4) << 30, s, d_err, fill, after));
    GDSW_TRY(read_err(d_err, s, "exact local Cholesky"));
    if (c->fp32) {
      float* a;
      GDSW_TRY(dalloc(c, &a, total));
      k_convert<float><<<grid_for(total, 256), 256, 0, s>>>(total, X, a);
      c->ainv = a;
    } else {
      double* a;
      GDSW_TRY(dalloc(c, &a, total));
      GDSW_CK(cudaMemcpyAsync(a, X, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
      c->ainv = a;
    }
    GDSW_CK(cudaGetLastError());
    GDSW_CK(cudaStreamSynchronize(s));
    c->stats.dense_local = total;
  }
  c->stats.setup_phase_seconds[6] = now_s() - t0;
  return GDSW_OK;
}

}  // namespace gdsw
