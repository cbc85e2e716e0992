// The preconditioner apply z = M^-1 r (Sec. III, Eq. 1) as four phases, the
// one-level branch and the coarse branch on two streams:
//
//  1. local:   one CTA per overlapping subdomain gathers r_s = R_s r into
//              shared memory and solves A_s z_s = r_s there: level-scheduled
//              substitution with the IC(k)/ILU(k) factors streamed as
//              per-level records by a producer warp (bulk copies into a ring),
//              the same from L2 without the ring, Jacobi sweeps, or the dense
//              inverse of the exact solver; z_s goes to the concatenated
//              local-solution buffer.
//  2. phiT:    partial products Phi_b^T r_b per chunk of a Phi block (a
//              subdomain interior or an interface component).
//  3. coarse:  c = sum of partials per coarse column (fixed order), then
//              y = A0^-1 c as a dense FP64 GEMV with the explicit inverse.
//  4. combine: every unknown is owned by exactly one Phi block; its thread sums
//              the overlapping local solutions in ascending subdomain order
//              (the deterministic scatter-add of sum_s R_s^T z_s) and adds
//              the prolongation (Phi y)_g, optionally fusing the PCG dots.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <type_traits>

#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace gdsw {

namespace {

// v = R_s r for one subdomain (m entries from base) by `nt` threads (this
// thread is `tid`): sixteen indices, then sixteen values, in flight per thread
// (each round costs two dependent global-memory latencies).
template <class T>
__device__ __forceinline__ void gather_sub(const double* __restrict__ r, const int* __restrict__ om_dofs,
                                           int base, int m, T* v, int tid, int nt) {
  constexpr int U = 16;
  for (int i0 = tid; i0 < m; i0 += U * nt) {
    int idx[U];
    uint64_t rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) idx[u] = i0 + u * nt < m ? om_dofs[base + i0 + u * nt] : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) rv[u] = idx[u] >= 0 ? load_bits(r, idx[u]) : 0ull;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * nt < m) v[i0 + u * nt] = narrow_bits<T>(rv[u]);
  }
}

// Level-scheduled substitution: the rows of a level are independent except
// within a node's group of E.grp consecutive rows, which one thread solves in
// the stored order.
template <class T>
__device__ __forceinline__ void tri_levels(const EllDev<T>& E, int s, T* v) {
  const int l0 = E.sub_lev[s], l1 = E.sub_lev[s + 1];
  const int G = E.grp;
  for (int l = l0; l < l1; ++l) {
    const int4 lv = E.lev[l];   // (first row, rows, width, first slot)
    for (int gt = threadIdx.x; gt * G < lv.y; gt += blockDim.x) {
      for (int d = 0; d < G; ++d) {
        const int t = gt * G + d;
        const int row = E.lrows[lv.x + t];
        T acc = v[row];
        const T* vals = E.val + lv.w + t;
        const uint16_t* cols = E.col + lv.w + t;
        for (int k = 0; k < lv.z; ++k) acc -= vals[int64_t(k) * lv.y] * v[cols[int64_t(k) * lv.y]];
        v[row] = acc * E.dinv[lv.x + t];
      }
    }
    __syncthreads();
  }
}

// Jacobi sweeps on T y = b (Sec. V-B3): y0 = D^-1 b, y_{k+1} = D^-1 (b - (T - D) y_k).
// b and the result share `b`; y0, y1 are work vectors of the CTA.
template <class T>
__device__ __forceinline__ void tri_jacobi(const EllDev<T>& E, int s, int sweeps, T* b, T* y0,
                                           T* y1) {
  const int l0 = E.sub_lev[s], l1 = E.sub_lev[s + 1];
  for (int l = l0; l < l1; ++l) {
    const int4 lv = E.lev[l];
    for (int t = threadIdx.x; t < lv.y; t += blockDim.x) {
      const int row = E.lrows[lv.x + t];
      y0[row] = b[row] * E.dinv[lv.x + t];
    }
  }
  __syncthreads();
  T* yo = y0;
  T* yn = y1;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int l = l0; l < l1; ++l) {
      const int4 lv = E.lev[l];
      for (int t = threadIdx.x; t < lv.y; t += blockDim.x) {
        const int row = E.lrows[lv.x + t];
        T acc = b[row];
        const T* vals = E.val + lv.w + t;
        const uint16_t* cols = E.col + lv.w + t;
        for (int k = 0; k < lv.z; ++k) acc -= vals[int64_t(k) * lv.y] * yo[cols[int64_t(k) * lv.y]];
        yn[row] = acc * E.dinv[lv.x + t];
      }
    }
    __syncthreads();
    T* tmp = yo; yo = yn; yn = tmp;
  }
  // result back into b
  for (int l = l0; l < l1; ++l) {
    const int4 lv = E.lev[l];
    for (int t = threadIdx.x; t < lv.y; t += blockDim.x) {
      const int row = E.lrows[lv.x + t];
      b[row] = yo[row];
    }
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(1024) k_local_tri(const double* __restrict__ r,
                                                   const int* __restrict__ om_ptr,
                                                   const int* __restrict__ om_dofs, EllDev<T> L,
                                                   EllDev<T> U, int jacobi, int sweeps,
                                                   T* __restrict__ zloc,
                                                   const KrylovScalars* __restrict__ ks, BatchGate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (ks != nullptr && ks->done) return;
  T* v = reinterpret_cast<T*>(smem_raw);
  const int s = blockIdx.x;
  if (gate_sub_off(gate, s)) return;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  gather_sub(r, om_dofs, base, m, v, threadIdx.x, blockDim.x);
  __syncthreads();
  if (!jacobi) {
    tri_levels(L, s, v);
    tri_levels(U, s, v);
  } else {
    T* y0 = v + m;
    T* y1 = v + 2 * m;
    tri_jacobi(L, s, sweeps, v, y0, y1);
    tri_jacobi(U, s, sweeps, v, y0, y1);
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) zloc[base + i] = v[i];
}

// Level-scheduled triangular solves streamed through shared memory.  The L
// levels and then the U levels of subdomain s are a sequence of records (one
// per level, 16-byte aligned, see the setup); a producer warp keeps S records
// in flight with bulk copies into a ring of stages, each stage tracked by
// mbarriers, while the consumer threads compute the current level from
// shared memory:
//     v[row] = (v[row] - sum_k val_k v[col_k]) * dinv
// Every wait is bounded by `wait_cycles`; a wait that runs out sets err[0],
// waits (bounded again) for the copies still in flight, and ends the CTA
// without writing z_s.

template <class T, class TS>
__device__ __forceinline__ T load_as(const TS* p, int i) { return T(p[i]); }
template <>
__device__ __forceinline__ float load_as<float, __half>(const __half* p, int i) { return __half2float(p[i]); }

// The four values of row t of a row-major record (16-byte aligned rows for
// FP32, 32 for FP64, 8 for FP16), widened to T.
template <class T, class TS>
__device__ __forceinline__ void load4(const TS* vals, int t, T* a);
template <>
__device__ __forceinline__ void load4<float, float>(const float* vals, int t, float* a) {
  const float4 q = reinterpret_cast<const float4*>(vals)[t];
  a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
}
template <>
__device__ __forceinline__ void load4<double, double>(const double* vals, int t, double* a) {
  const double2 q0 = reinterpret_cast<const double2*>(vals)[2 * t];
  const double2 q1 = reinterpret_cast<const double2*>(vals)[2 * t + 1];
  a[0] = q0.x; a[1] = q0.y; a[2] = q1.x; a[3] = q1.y;
}
template <>
__device__ __forceinline__ void load4<float, __half>(const __half* vals, int t, float* a) {
  const uint2 q = reinterpret_cast<const uint2*>(vals)[t];
  const __half2 h0 = *reinterpret_cast<const __half2*>(&q.x);
  const __half2 h1 = *reinterpret_cast<const __half2*>(&q.y);
  const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
  a[0] = f0.x; a[1] = f0.y; a[2] = f1.x; a[3] = f1.y;
}

// Row update of one level: TPR threads per row split the row's entries and
// add their partial sums with shuffles; short rows (TPR = 1) are unrolled.
// TS is the storage type of the record values (T, or FP16 applied in FP32).
template <class T, class TS, int TPR>
__device__ __forceinline__ void level_rows(const unsigned char* rec, T* v, const int NT, const int G) {
  const int4 hdr = *reinterpret_cast<const int4*>(rec);
  const int4 hdr1 = *reinterpret_cast<const int4*>(rec + 16);
  const int nr = hdr.x, K = hdr.y;          // rows, stored width
  const int layout = hdr1.y & 0xff;         // 0 column-major, 1 row-major by 4, 2 by node
  const uint16_t* lrows = reinterpret_cast<const uint16_t*>(rec + 32);
  const TS* dinv = reinterpret_cast<const TS*>(rec + 32 + ((2 * nr + 15) & ~15));
  const TS* vals = reinterpret_cast<const TS*>(rec + hdr.z);
  const uint16_t* cols = reinterpret_cast<const uint16_t*>(rec + hdr.w);
  const TS* inn = reinterpret_cast<const TS*>(rec + hdr1.x);
  if (layout == 2) {
    // by node: the G rows' couplings to other nodes summed at once, then the
    // rows of the node solved in order with the in-node coefficients
    const int sub = TPR == 1 ? 0 : threadIdx.x % TPR;
    const int groups = NT / TPR;
    const int ngr = nr / G;
    for (int round = 0; round < ngr; round += groups) {
      const int gt = round + threadIdx.x / TPR;
      const bool valid = gt < ngr;
      T part[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        part[d] = T(0);
        if (valid && d < G) {
          const int t = gt * G + d;
          for (int k = sub; k < K; k += TPR)
            part[d] = fma(load_as<T, TS>(vals, k * nr + t), v[cols[k * nr + t]], part[d]);
        }
      }
      if (TPR > 1) {
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
          for (int o = TPR / 2; o > 0; o >>= 1) part[d] += __shfl_down_sync(0xffffffffu, part[d], o, TPR);
      }
      if (valid && sub == 0) {
        T y[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          if (d < G) {
            const int t = gt * G + d;
            const int row = lrows[t];
            T acc = v[row] - part[d];
#pragma unroll
            for (int q = 0; q < 3; ++q)
              if (q < d) acc = fma(-load_as<T, TS>(inn, t * (G - 1) + q), y[q], acc);
            y[d] = acc * load_as<T, TS>(dinv, t);
            v[row] = y[d];
          }
        }
      }
    }
  } else if (TPR == 1) {
    for (int t = threadIdx.x; t < nr; t += NT) {
      const int row = lrows[t];
      T acc = v[row];
      if (layout == 1) {
        // one vector load of the four columns and one of the four values
        const ushort4 c4 = reinterpret_cast<const ushort4*>(cols)[t];
        T a[4];
        load4<T, TS>(vals, t, a);
        acc = fma(-a[0], v[c4.x], acc);
        acc = fma(-a[1], v[c4.y], acc);
        acc = fma(-a[2], v[c4.z], acc);
        acc = fma(-a[3], v[c4.w], acc);
      } else {
        for (int k = 0; k < K; ++k) acc = fma(-load_as<T, TS>(vals, k * nr + t), v[cols[k * nr + t]], acc);
      }
      v[row] = acc * load_as<T, TS>(dinv, t);
    }
  } else {
    const int sub = threadIdx.x % TPR;
    const int groups = NT / TPR;
    // every thread runs the same number of rounds, so the shuffles stay convergent
    for (int round = 0; round < nr; round += groups) {
      const int t = round + threadIdx.x / TPR;
      T part = T(0);
      if (t < nr) {
        if (layout == 1) {
          for (int k = sub; k < 4; k += TPR) part = fma(load_as<T, TS>(vals, t * 4 + k), v[cols[t * 4 + k]], part);
        } else {
          for (int k = sub; k < K; k += TPR) part = fma(load_as<T, TS>(vals, k * nr + t), v[cols[k * nr + t]], part);
        }
      }
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o, TPR);
      if (t < nr && sub == 0) {
        const int row = lrows[t];
        v[row] = (v[row] - part) * load_as<T, TS>(dinv, t);
      }
    }
  }
}

// The pipelined local solve runs NT consumer threads (64 to 512, chosen at
// setup) that update the rows, plus one producer warp that only streams the
// level records into the ring (at most 544 threads, so the compiler may give a
// thread up to 112 registers instead of the 64 that 1024 threads would leave).
constexpr int kPipeMaxThreads = 544;

// Barrier of the `nt` consumer threads only (named barrier 1), every warp
// arriving whole at the same instruction.
__device__ __forceinline__ void consumers_sync_aligned(int nt) {
  asm volatile("barrier.cta.sync.aligned 1, %0;" ::"r"(nt) : "memory");
}

// Barrier of the `nt` consumer threads only (named barrier 1), returning the
// OR of `pred` over them.
__device__ __forceinline__ bool consumers_sync_or(bool pred, int nt) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.cta.red.or.pred p, 1, %2, q;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(out)
      : "r"(static_cast<uint32_t>(pred)), "r"(nt)
      : "memory");
  return out != 0;
}

// v = R_s r from indices already staged in shared memory (`idx`: this
// subdomain's slice of the overlap map), sixteen values in flight per thread.
// For FP32 vectors `idx` and `v` share their words: each thread reads and
// writes only its own positions.  For FP64 `idx` sits in the upper half of
// the vector's space, and a barrier between the index reads and the value
// writes of each round keeps a value from overwriting an index still to be
// read (the values of a round land below the indices of every later round).
template <class T>
__device__ __forceinline__ void gather_staged(const double* __restrict__ r, const int* idx, T* v, int m,
                                              int nt) {
  constexpr int U = 16;
  const int tid = threadIdx.x;
  for (int i0 = 0; i0 < m; i0 += U * nt) {
    uint64_t rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + tid + u * nt;
      rv[u] = i < m ? load_bits(r, idx[i]) : 0ull;
    }
    if (sizeof(T) == 8) consumers_sync_or(false, nt);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + tid + u * nt;
      if (i < m) v[i] = narrow_bits<T>(rv[u]);
    }
  }
}

// Shared memory of the pipelined solve's local vector: m values plus the room
// the staged overlap indices need (an aligned start and up to three words on
// either side of the subdomain's slice).
inline size_t pipe_vector_bytes(int max_m, size_t es) { return (size_t(max_m) * es + 48 + 15) & ~size_t(15); }

// Producer warp of the pipelined local solves: lane 0 first copies the
// subdomain's overlap indices (om_dofs[first, first + cnt), one bulk copy into
// idx_dst, completing on gbar); the lanes fetch the pack offsets and sizes 32
// at a time, lane 0 waits for free stages and issues the copies, and keeps
// `prefetch_bytes` of the subdomain's records beyond the ring on their way
// into L2.  Every copy issued has landed before it returns.
template <int S>
__device__ __forceinline__ void pipe_producer(const int* __restrict__ om_dofs, int first, int cnt,
                                              unsigned char* idx_dst, uint64_t* gbar,
                                              const uint32_t* __restrict__ rec_off16,
                                              const uint32_t* __restrict__ rec_bytes, int r0, int nrec,
                                              const uint8_t* __restrict__ stream, unsigned char* stages,
                                              int stage_bytes, uint64_t* full, uint64_t* empty, int* err,
                                              long long wait_cycles, int stall_test, int prefetch_bytes) {
  const int lane = threadIdx.x & 31;
  if (lane == 0 && cnt > 0) {
    mbar_expect_tx(gbar, unsigned(cnt) * 4u);
    bulk_g2s(idx_dst, om_dofs + first, unsigned(cnt) * 4u, gbar);
  }
  int last[S];
#pragma unroll
  for (int j = 0; j < S; ++j) last[j] = -1;
  uint32_t my_off = 0, my_nb = 0;
  // end of the subdomain's record bytes, and how far the L2 prefetch reached
  size_t pf_end = 0, pf = 0;
  if (nrec > 0 && prefetch_bytes > 0) {
    pf_end = size_t(rec_off16[r0 + nrec - 1]) * 16 + rec_bytes[r0 + nrec - 1];
    pf = size_t(rec_off16[r0]) * 16;
  }
  for (int j = 0; j < nrec; ++j) {
    if ((j & 31) == 0 && j + lane < nrec) {
      my_off = rec_off16[r0 + j + lane];
      my_nb = rec_bytes[r0 + j + lane];
    }
    const uint32_t off16 = __shfl_sync(0xffffffffu, my_off, j & 31);
    const uint32_t nb = __shfl_sync(0xffffffffu, my_nb, j & 31);
    const int st = j % S;
    int stop = 0;
    if (lane == 0) {
      if (j >= S && !mbar_wait_bounded(&empty[st], ((j / S) - 1) & 1, wait_cycles)) {
        atomicOr(err, 1);    // the consumers stopped (their own wait ran out)
        stop = 1;
      } else if (!(stall_test && j == 1)) {
        // (failure test: record 1 is never copied, so the consumers' wait
        // for it runs out; its `full` barrier is a flag that nothing sets)
        fence_proxy_async_smem();
        mbar_expect_tx(&full[st], nb);
        bulk_g2s(stages + size_t(st) * stage_bytes, stream + size_t(off16) * 16, nb, &full[st]);
        last[st] = j;
      }
      if (prefetch_bytes > 0 && !stop) {
        // records up to `prefetch_bytes` past this pack, in pieces of at
        // most 16 KB, start their way into L2 (16-byte aligned: records are)
        const size_t here = size_t(off16) * 16 + nb;
        if (pf < here) pf = here;
        const size_t want = here + size_t(prefetch_bytes) < pf_end ? here + size_t(prefetch_bytes) : pf_end;
        while (pf < want) {
          const size_t piece = want - pf < 16384 ? want - pf : 16384;
          bulk_prefetch_l2(stream + pf, static_cast<unsigned>(piece));
          pf += piece;
        }
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) break;
  }
  if (lane != 0) return;
  // every copy issued has landed before the CTA's shared memory can go away
  // (waited for with at least the default bound, however short the caller's)
  const long long drain = wait_cycles > kDefaultWaitCycles ? wait_cycles : kDefaultWaitCycles;
#pragma unroll
  for (int st = 0; st < S; ++st)
    if (last[st] >= 0) mbar_wait_bounded(&full[st], (last[st] / S) & 1, drain);
  if (cnt > 0) mbar_wait_bounded(gbar, 0, drain);
}

// z_s = (L U)^-1 r_s for every subdomain s (one CTA each), level by level.
// The producer warp copies the level records of subdomain s, several small
// consecutive ones packed into one bulk copy, into a ring of S stages
// (full[st] completes when a pack has landed, empty[st] when every consumer
// warp is done with it); the consumers wait for a pack, update the rows of its
// levels in shared memory with one barrier per level, and release the stage.
// The copy issue is off the consumers' path.
template <class T, class TS, int S, int TPR>
__global__ void __launch_bounds__(kPipeMaxThreads, 1) k_local_pipe(const double* __restrict__ r,
                                                             const int* __restrict__ om_ptr,
                                                             const int* __restrict__ om_dofs,
                                                             const int* __restrict__ rec_ptr,
                                                             const uint32_t* __restrict__ rec_off16,
                                                             const uint32_t* __restrict__ rec_bytes,
                                                             const uint8_t* __restrict__ stream, int stage_bytes,
                                                             T* __restrict__ zloc,
                                                             const KrylovScalars* __restrict__ ks, int* err,
                                                             long long wait_cycles, int grp, int stall_test,
                                                             int prefetch_bytes, BatchGate gate) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[S];
  __shared__ __align__(8) uint64_t empty[S];
  __shared__ __align__(8) uint64_t gbar;    // the staged overlap indices have landed
  __shared__ int s_fail;                     // a consumer's wait ran out
  if (ks != nullptr && ks->done) return;
  const int s = blockIdx.x;
  if (gate_sub_off(gate, s)) return;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  const int r0 = rec_ptr[s], nrec = rec_ptr[s + 1] - r0;
  unsigned char* stages = smem_raw;
  unsigned char* vreg = smem_raw + size_t(S) * stage_bytes;
  // the overlap indices om_dofs[base - off, base - off + cnt) arrive by one
  // bulk copy (16-byte aligned source and size); position i's index is then
  // word off + i of the staged slice
  const int off = base & 3;
  const int cnt = m > 0 ? (off + m + 3) & ~3 : 0;
  const int m4 = (m + 3) & ~3;
  unsigned char* idx_dst = sizeof(T) == 4 ? vreg : vreg + size_t(4) * m4;
  const int* idx = reinterpret_cast<const int*>(idx_dst) + off;
  T* v = sizeof(T) == 4 ? reinterpret_cast<T*>(vreg) + off : reinterpret_cast<T*>(vreg);
  const int nt = blockDim.x - 32;            // consumer threads
  if (threadIdx.x == 0) {
    for (int j = 0; j < S; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], nt / 32);         // one arrival per consumer warp
    }
    mbar_init(&gbar, 1);
    s_fail = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (int(threadIdx.x) >= nt) {
    pipe_producer<S>(om_dofs, base - off, cnt, idx_dst, &gbar, rec_off16, rec_bytes, r0, nrec, stream, stages,
                     stage_bytes, full, empty, err, wait_cycles, stall_test, prefetch_bytes);
    return;
  }
  // ---- consumer warps ----
  {
    const bool ok = m == 0 || mbar_wait_bounded(&gbar, 0, wait_cycles);
    if (consumers_sync_or(!ok, nt)) {
      if (threadIdx.x == 0) atomicOr(err, 1);
      return;
    }
  }
  gather_staged(r, idx, v, m, nt);
  consumers_sync_aligned(nt);
  volatile int* fail = &s_fail;
  for (int i = 0; i < nrec; ++i) {
    const int st = i % S;
    // each thread waits for the pack itself, then all agree that it has
    // landed before any reads it: a wait that runs out raises the CTA's
    // failure flag before the barrier, and every thread reads it after
    if (!mbar_wait_bounded(&full[st], (i / S) & 1, wait_cycles)) *fail = 1;
    consumers_sync_aligned(nt);
    if (*fail) {
      if (threadIdx.x == 0) atomicOr(err, 1);
      return;
    }
    // the stage holds a pack of consecutive level records (their count in the
    // first header, each record's size in its own); one barrier per level,
    // after its last record
    const unsigned char* rec = stages + size_t(st) * stage_bytes;
    const int count = reinterpret_cast<const int*>(rec)[7];
    for (int q = 0; q < count; ++q) {
      const unsigned char* next = rec + reinterpret_cast<const int*>(rec)[6];
      const bool level_end = (reinterpret_cast<const int*>(rec)[5] & kRecLevelEnd) != 0;
      level_rows<T, TS, TPR>(rec, v, nt, grp);
      // each warp releases the stage as soon as its lanes are done reading it
      if (q + 1 == count) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0 && i + S < nrec) mbar_arrive(&empty[st]);
      }
      if (level_end) consumers_sync_aligned(nt);
      rec = next;
    }
  }
  for (int i = threadIdx.x; i < m; i += nt) zloc[base + i] = v[i];
}

// ---- level-scheduled solve from row programs ----
//
// One CTA of kStepRows threads per subdomain executes the subdomain's row
// program (its L levels, then its U levels, each level cut into steps of at
// most kStepRows rows; thread t takes row t of a step).  Thread t's
// instruction of a step -- A: float4 {a0, a1, a2, inverse diagonal}, C: uint2
// {c0 | c1 << 16, c2 | row << 16} -- comes with its own cp.async copies into
// its slot of a D-step ring, issued D - 1 steps ahead; no thread waits on
// another for data, so the only synchronisation is one CTA barrier at the end
// of each level, and there is no spin-wait that could run out.  Per row: acc
// = z[row]; acc -= a_k z[c_k] (k = 0, 1, 2, slot order); z[row] = acc *
// inverse diagonal -- the arithmetic of the row-major records, so the result
// equals k_local_pipe's.  The overlap indices arrive the same way (16-byte
// copies of the 4-word-padded slice) before r is gathered.
//
// (Bulk copies of whole steps by one thread into mbarrier-tracked slots were
// measured slower here: every thread then polls the barrier, and the refills
// wait for the level barriers.)
template <int D>
__global__ void __launch_bounds__(kStepRows, 4) k_local_steps(const double* __restrict__ r,
                                                           const int* __restrict__ om_ptr,
                                                           const int* __restrict__ om_dofs,
                                                           const int* __restrict__ step_ptr,
                                                           const int2* __restrict__ steps,
                                                           const float4* __restrict__ prog_a,
                                                           const uint2* __restrict__ prog_c,
                                                           int step_max, float* __restrict__ zloc,
                                                           const KrylovScalars* __restrict__ ks, BatchGate gate) {
  static_assert(D >= 3, "the ring refills the slot read one step earlier");
  constexpr int NT = kStepRows;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (ks != nullptr && ks->done) return;
  const int s = blockIdx.x;
  if (gate_sub_off(gate, s)) return;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  const int st0 = step_ptr[s], nst = step_ptr[s + 1] - st0;
  const int t = threadIdx.x;
  float4* ring_a = reinterpret_cast<float4*>(smem_raw);
  uint2* ring_c = reinterpret_cast<uint2*>(smem_raw + size_t(D) * NT * 16);
  int2* stp = reinterpret_cast<int2*>(smem_raw + size_t(D) * NT * 24);
  unsigned char* vreg = smem_raw + size_t(D) * NT * 24 + ((size_t(step_max) * 8 + 15) & ~size_t(15));
  const int off = base & 3;
  const int cnt = m > 0 ? (off + m + 3) & ~3 : 0;
  const int* idx = reinterpret_cast<const int*>(vreg) + off;
  float* v = reinterpret_cast<float*>(vreg) + off;
  // group 0: the overlap indices; groups 1..D: the first D steps
  for (int q = t; q < cnt / 4; q += NT) cp_async16(vreg + 16 * q, om_dofs + (base - off) + 4 * q);
  cp_async_commit();
  for (int d = 0; d < D; ++d) {
    if (d < nst) {
      const int2 sd = steps[st0 + d];
      if (t < (sd.y & 0xffff)) {
        cp_async16(&ring_a[d * NT + t], prog_a + sd.x + t);
        cp_async8(&ring_c[d * NT + t], prog_c + sd.x + t);
      }
    }
    cp_async_commit();
  }
  for (int q = t; q < nst; q += NT) stp[q] = steps[st0 + q];
  cp_async_wait<D>();
  __syncthreads();
  gather_staged(r, idx, v, m, NT);
  // the first step's instruction into registers; each later one is read
  // before the previous step's barrier, so a step starts from registers
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  uint2 cc = make_uint2(0u, 0u);
  if (nst > 0) {
    cp_async_wait<D - 1>();
    if (t < (stp[0].y & 0xffff)) {
      a = ring_a[t];
      cc = ring_c[t];
    }
  }
  __syncthreads();
  // the steps go D at a time, unrolled, so every ring slot is a compile-time
  // offset from this thread's slot 0; the step table entries of the current,
  // refilled and next steps are read once each
  const float4* pa = prog_a + t;
  const uint2* pc = prog_c + t;
  float4* ra = ring_a + t;
  uint2* rc = ring_c + t;
  int2 sd_next = nst > 0 ? stp[0] : make_int2(0, 0);
  for (int i0 = 0; i0 < nst; i0 += D) {
#pragma unroll
    for (int u = 0; u < D; ++u) {
      const int i = i0 + u;
      if (i >= nst) break;
      const int2 sd = sd_next;
      // refill the slot read during the previous step (its values are already
      // in registers, so the copy cannot overtake the read) with step i - 1 + D
      if (i > 0) {
        const int j = i - 1 + D;
        if (j < nst) {
          const int2 sn = stp[j];
          const int slot = (u + D - 1) % D;   // a constant once unrolled
          if (t < (sn.y & 0xffff)) {
            cp_async16(ra + slot * NT, pa + sn.x);
            cp_async8(rc + slot * NT, pc + sn.x);
          }
        }
        cp_async_commit();
      }
      if (t < (sd.y & 0xffff)) {
        const int row = cc.y >> 16;
        float acc = v[row];
        acc = fmaf(-a.x, v[cc.x & 0xffff], acc);
        acc = fmaf(-a.y, v[cc.x >> 16], acc);
        acc = fmaf(-a.z, v[cc.y & 0xffff], acc);
        v[row] = acc * a.w;
      }
      if (i + 1 < nst) {
        // step i + 1's group: D + i groups of steps committed, i + 2 of them done
        cp_async_wait<D - 2>();
        sd_next = stp[i + 1];
        if (t < (sd_next.y & 0xffff)) {
          const int slot = (u + 1) % D;
          a = ra[slot * NT];
          cc = rc[slot * NT];
        }
      }
      if (sd.y >> 16) __syncthreads();
    }
  }
  for (int q = t; q < m; q += NT) zloc[base + q] = v[q];
}

// ---- level-scheduled solve from node programs (three unknowns per node) ----
//
// One CTA of NT threads per subdomain; LPN lanes (2, 4 or 8) per node.  The
// pieces of the subdomain's node program (see the setup's node programs) come
// by bulk copies, issued by one thread, into a ring of S (at most kNodeSlots)
// slots (an mbarrier per slot completing on the bytes, waits bounded), S
// pieces ahead.  Per node: each lane sums VW = 8 / LPN consecutive columns of
// every chunk of eight of the node's off-node columns, for the three rows at
// once (z at a column is read once for all three; columns and values by
// vector loads, a node's lanes reading each chunk contiguously), the lanes' partial
// sums meet in a shuffle tree, and the node's first lane solves the three rows
// in order with the in-node coefficients; warps without a node in the level
// go straight to the barrier that ends the piece, after which the issuing
// thread refills the slot.  A wait that runs out sets the failure flag; the
// threads leave together at the next barrier, the issuing thread lets its
// copies land, and z_s is not written.
constexpr int kNodeSlots = 6;

// The lane's share of a node's sums: chunks of eight columns, the lane taking
// VW consecutive columns of each (lane * VW onward), so the LPN = 8 / VW lanes
// of a node read each chunk's columns and values contiguously.
template <int VW>
struct NodeVec;
template <>
struct NodeVec<1> {
  __device__ static void sums(const uint16_t* cn, const float* vn, int K, int j0, const float* v, float& s0,
                              float& s1, float& s2) {
#pragma unroll 4
    for (int j = j0; j < K; j += 8) {
      const float x = v[cn[j]];
      s0 = fmaf(vn[j], x, s0);
      s1 = fmaf(vn[K + j], x, s1);
      s2 = fmaf(vn[2 * K + j], x, s2);
    }
  }
};
template <>
struct NodeVec<2> {
  __device__ static void sums(const uint16_t* cn, const float* vn, int K, int j0, const float* v, float& s0,
                              float& s1, float& s2) {
#pragma unroll 2
    for (int j = j0; j < K; j += 8) {
      const uint32_t c = *reinterpret_cast<const uint32_t*>(cn + j);
      const float x0 = v[c & 0xffffu], x1 = v[c >> 16];
      const float2 a = *reinterpret_cast<const float2*>(vn + j);
      const float2 b = *reinterpret_cast<const float2*>(vn + K + j);
      const float2 d = *reinterpret_cast<const float2*>(vn + 2 * K + j);
      s0 = fmaf(a.y, x1, fmaf(a.x, x0, s0));
      s1 = fmaf(b.y, x1, fmaf(b.x, x0, s1));
      s2 = fmaf(d.y, x1, fmaf(d.x, x0, s2));
    }
  }
};
template <>
struct NodeVec<4> {
  __device__ static void sums(const uint16_t* cn, const float* vn, int K, int j0, const float* v, float& s0,
                              float& s1, float& s2) {
    for (int j = j0; j < K; j += 8) {
      const uint2 c = *reinterpret_cast<const uint2*>(cn + j);
      const float x0 = v[c.x & 0xffffu], x1 = v[c.x >> 16], x2 = v[c.y & 0xffffu], x3 = v[c.y >> 16];
      const float4 a = *reinterpret_cast<const float4*>(vn + j);
      const float4 b = *reinterpret_cast<const float4*>(vn + K + j);
      const float4 d = *reinterpret_cast<const float4*>(vn + 2 * K + j);
      s0 = fmaf(a.w, x3, fmaf(a.z, x2, fmaf(a.y, x1, fmaf(a.x, x0, s0))));
      s1 = fmaf(b.w, x3, fmaf(b.z, x2, fmaf(b.y, x1, fmaf(b.x, x0, s1))));
      s2 = fmaf(d.w, x3, fmaf(d.z, x2, fmaf(d.y, x1, fmaf(d.x, x0, s2))));
    }
  }
};

template <int NT, int LPN>
__global__ void __launch_bounds__(NT, 1) k_local_nodes(const double* __restrict__ r,
                                                       const int* __restrict__ om_ptr,
                                                       const int* __restrict__ om_dofs,
                                                       const int* __restrict__ node_ptr,
                                                       const int4* __restrict__ pieces,
                                                       const uint8_t* __restrict__ stream, int S,
                                                       int slot_bytes, float* __restrict__ zloc,
                                                       const KrylovScalars* __restrict__ ks, int* err,
                                                       long long wait_cycles, int stall_test, BatchGate gate) {
  static_assert(LPN == 2 || LPN == 4 || LPN == 8, "2, 4 or 8 lanes per node");
  // K is a multiple of 8: a node's LPN lanes take VW = 8 / LPN columns of
  // each chunk of eight
  constexpr int VW = 8 / LPN;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kNodeSlots];
  __shared__ __align__(8) uint64_t gbar;
  __shared__ int s_fail;
  if (ks != nullptr && ks->done) return;
  const int s = blockIdx.x;
  if (gate_sub_off(gate, s)) return;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  const int p0 = node_ptr[s], np = node_ptr[s + 1] - p0;
  unsigned char* ring = smem_raw;
  unsigned char* vreg = smem_raw + size_t(S) * slot_bytes;
  const int off = base & 3;
  const int cnt = m > 0 ? (off + m + 3) & ~3 : 0;
  const int* idx = reinterpret_cast<const int*>(vreg) + off;
  float* v = reinterpret_cast<float*>(vreg) + off;
  const int t = threadIdx.x, lane = t % LPN, group = t / LPN;
  constexpr int NG = NT / LPN;
  constexpr int kWarpGroups = 32 / LPN;
  const int warp_first = (t >> 5) * kWarpGroups;
  const bool withhold = stall_test && s == 0;
  // the copies are issued by the last thread, whose warp has nodes only in
  // the widest levels; it holds the table entry of the next piece in a
  // register, loaded a level ahead
  constexpr int kIssuer = NT - 1;
  int issued = 0;
  int4 nxt = make_int4(0, 0, 0, 0);
  auto issue = [&](int j) {
    const unsigned bytes = unsigned(nxt.y + 15) & ~15u;
    mbar_expect_tx(&full[j % S], bytes);
    bulk_g2s(ring + size_t(j % S) * slot_bytes, stream + size_t(nxt.x) * 16, bytes, &full[j % S]);
    if (j + 1 < np) nxt = pieces[p0 + j + 1];
  };
  if (t == kIssuer) {
    for (int d = 0; d < S; ++d) mbar_init(&full[d], 1);
    mbar_init(&gbar, 1);
    s_fail = 0;
    fence_mbar_init();
    if (cnt > 0) {
      mbar_expect_tx(&gbar, unsigned(cnt) * 4u);
      bulk_g2s(vreg, om_dofs + (base - off), unsigned(cnt) * 4u, &gbar);
    }
    if (np > 0) nxt = pieces[p0];
    issued = min(S, np);
    for (int j = 0; j < issued; ++j) {
      if (withhold && j == 0) {
        if (1 < np) nxt = pieces[p0 + 1];
      } else {
        issue(j);
      }
    }
  }
  __syncthreads();
  if (cnt > 0 && !mbar_wait_bounded(&gbar, 0, wait_cycles)) s_fail = 1;
  __syncthreads();
  bool failed = s_fail != 0;
  if (!failed) gather_staged(r, idx, v, m, NT);
  __syncthreads();
  int waited = -1;                           // last piece whose copy this thread saw land
  int i = 0, slot = 0;
  unsigned phase = 0;
  for (; i < np && !failed; ++i) {
    if (!mbar_wait_bounded(&full[slot], phase, wait_cycles)) {
      s_fail = 1;
    } else {
      waited = i;
      const unsigned char* pc = ring + size_t(slot) * slot_bytes;
      const int4 hdr = *reinterpret_cast<const int4*>(pc);
      const int N = hdr.x & 0xffff, K = hdr.y;
      const bool upper = (hdr.x >> 16) != 0;    // U sweep: the node's rows solved last to first
      const uint16_t* nodes = reinterpret_cast<const uint16_t*>(pc + 16);
      const float4* coef = reinterpret_cast<const float4*>(pc + 16 + ((2 * N + 15) & ~15));
      const uint16_t* cols = reinterpret_cast<const uint16_t*>(pc + hdr.z);
      const float* vals = reinterpret_cast<const float*>(pc + hdr.w);
      // rounds of NG nodes; a warp whose first node is past the level's end
      // has none in this round or later ones (warp-uniform exit)
      for (int round = 0; round + warp_first < N; round += NG) {
        const int n = round + group;
        const bool valid = n < N;
        const bool solver = valid && lane == 0;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        // the solving lane's operands (its own rows: no other node writes them
        // in this level), loaded before the sums so their latency overlaps
        int ra = 0, rb = 0, rc = 0;
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f), cc = d;
        float va = 0.f, vb = 0.f, vc = 0.f;
        if (solver) {
          const int g = nodes[n];
          // the row of solve step q: 3g + q in the L sweep, 3g + 2 - q in the U sweep
          ra = upper ? 3 * g + 2 : 3 * g;
          rb = 3 * g + 1;
          rc = upper ? 3 * g : 3 * g + 2;
          d = coef[2 * n];
          cc = coef[2 * n + 1];
          va = v[ra];
          vb = v[rb];
          vc = v[rc];
        }
        if (valid) NodeVec<VW>::sums(cols + size_t(n) * K, vals + size_t(n) * 3 * K, K, lane * VW, v, s0, s1, s2);
#pragma unroll
        for (int o = LPN / 2; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o, LPN);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o, LPN);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o, LPN);
        }
        if (solver) {
          // coefficients: d = {1/d0, 1/d1, 1/d2, c10}, cc = {c20, c21, -, -}
          const float y0 = (va - s0) * d.x;
          const float y1 = (vb - s1 - d.w * y0) * d.y;
          const float y2 = (vc - s2 - cc.x * y0 - cc.y * y1) * d.z;
          v[ra] = y0;
          v[rb] = y1;
          v[rc] = y2;
        }
      }
    }
    __syncthreads();
    failed = s_fail != 0;
    if (t == kIssuer && !failed) {
      const int lim = min(np, i + 1 + S);
      if (issued < lim) fence_proxy_async_smem();
      for (; issued < lim; ++issued) issue(issued);
    }
    if (++slot == S) {
      slot = 0;
      phase ^= 1u;
    }
  }
  if (failed) {
    if (t == kIssuer) {
      atomicOr(err, 1);
      for (int j = waited + 1; j < issued; ++j)
        if (!(withhold && j == 0)) mbar_wait_bounded(&full[j % S], (j / S) & 1, wait_cycles);
    }
    return;
  }
  for (int q = t; q < m; q += NT) zloc[base + q] = v[q];
}

// Shared memory of k_local_steps with D slots.
inline size_t steps_smem_bytes(int D, int step_max, int max_m) {
  return size_t(D) * kStepRows * 24 + ((size_t(step_max) * 8 + 15) & ~size_t(15)) + pipe_vector_bytes(max_m, 4);
}

// Shared memory of k_local_nodes with S ring slots.
inline size_t nodes_smem_bytes(int S, int slot_bytes, int max_m) {
  return size_t(S) * slot_bytes + pipe_vector_bytes(max_m, 4);
}

// ---- level-scheduled solve without a barrier per level ----
//
// The same records and producer as k_local_pipe, but the consumers meet at no
// barrier between levels: every row waits only for the rows it reads.  A byte
// per local row (in shared memory) says how far that row's value has got: 0
// the right-hand side, 1 final after the L sweep, 2 final after the U sweep.
// A row of sweep `phase` spins until every column it reads is flagged
// `phase`, updates its value, fences (CTA scope) and sets its own flag.  Each
// thread takes its rows in record order, and a row reads only rows of earlier
// records, so the earliest unfinished row can always proceed.  One barrier
// separates the two sweeps (the U sweep overwrites values the L sweep reads).
// Every spin is bounded; a wait that runs out sets the CTA's failure flag and
// err[0], after which every thread skips the remaining work but still meets
// the two barriers, and z_s is not written.

__device__ __forceinline__ void fence_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }

// Barrier of the `nt` consumer threads (named barrier 1), not .aligned: the
// threads of a warp may arrive from different places (a thread whose wait ran
// out meets the sweep barrier at the end of its loop).
__device__ __forceinline__ void consumers_sync(int nt) {
  asm volatile("barrier.cta.sync 1, %0;" ::"r"(nt) : "memory");
}

// Spins until flags[c] >= phase; false when `cycles` pass first or the CTA
// has failed.
__device__ __forceinline__ bool wait_row(const volatile unsigned char* flags, int c, int phase,
                                         long long cycles, const volatile int* fail) {
  if (flags[c] >= phase) return true;
  const long long t0 = clock64();
  for (;;) {
    if (flags[c] >= phase) return true;
    if (*fail) return false;
    if (clock64() - t0 > cycles) return false;
  }
}

// The rows of one level record for sweep `phase`; false when a wait ran out.
template <class T, class TS>
__device__ __forceinline__ bool sf_record(const unsigned char* rec, T* v, unsigned char* flags, int phase, int nt,
                                          int G, long long cycles, const volatile int* fail) {
  const int4 hdr = *reinterpret_cast<const int4*>(rec);
  const int4 hdr1 = *reinterpret_cast<const int4*>(rec + 16);
  const int nr = hdr.x, K = hdr.y;
  const int layout = hdr1.y & 0xff;
  const uint16_t* lrows = reinterpret_cast<const uint16_t*>(rec + 32);
  const TS* dinv = reinterpret_cast<const TS*>(rec + 32 + ((2 * nr + 15) & ~15));
  const TS* vals = reinterpret_cast<const TS*>(rec + hdr.z);
  const uint16_t* cols = reinterpret_cast<const uint16_t*>(rec + hdr.w);
  const TS* inn = reinterpret_cast<const TS*>(rec + hdr1.x);
  volatile unsigned char* vf = flags;
  if (layout == 1) {
    for (int t = threadIdx.x; t < nr; t += nt) {
      const int row = lrows[t];
      const ushort4 c4 = reinterpret_cast<const ushort4*>(cols)[t];
      // padding entries point at the row itself (value 0): nothing to wait for
      if ((c4.x != row && !wait_row(vf, c4.x, phase, cycles, fail)) ||
          (c4.y != row && !wait_row(vf, c4.y, phase, cycles, fail)) ||
          (c4.z != row && !wait_row(vf, c4.z, phase, cycles, fail)) ||
          (c4.w != row && !wait_row(vf, c4.w, phase, cycles, fail)))
        return false;
      fence_cta();
      T a[4];
      load4<T, TS>(vals, t, a);
      T acc = v[row];
      acc = fma(-a[0], v[c4.x], acc);
      acc = fma(-a[1], v[c4.y], acc);
      acc = fma(-a[2], v[c4.z], acc);
      acc = fma(-a[3], v[c4.w], acc);
      v[row] = acc * load_as<T, TS>(dinv, t);
      fence_cta();
      vf[row] = static_cast<unsigned char>(phase);
    }
  } else if (layout == 0) {
    for (int t = threadIdx.x; t < nr; t += nt) {
      const int row = lrows[t];
      for (int k = 0; k < K; ++k) {
        const int c = cols[k * nr + t];
        if (c != row && !wait_row(vf, c, phase, cycles, fail)) return false;
      }
      fence_cta();
      T acc = v[row];
      for (int k = 0; k < K; ++k) acc = fma(-load_as<T, TS>(vals, k * nr + t), v[cols[k * nr + t]], acc);
      v[row] = acc * load_as<T, TS>(dinv, t);
      fence_cta();
      vf[row] = static_cast<unsigned char>(phase);
    }
  } else {
    // by node: the G rows' couplings to other nodes (padding points at the
    // row itself), then the in-node triangle in order by this thread
    const int ngr = nr / G;
    for (int gt = threadIdx.x; gt < ngr; gt += nt) {
      for (int d = 0; d < G; ++d) {
        const int t = gt * G + d;
        const int row = lrows[t];
        for (int k = 0; k < K; ++k) {
          const int c = cols[k * nr + t];
          if (c != row && !wait_row(vf, c, phase, cycles, fail)) return false;
        }
      }
      fence_cta();
      T y[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (d < G) {
          const int t = gt * G + d;
          const int row = lrows[t];
          T part = T(0);
          for (int k = 0; k < K; ++k) part = fma(load_as<T, TS>(vals, k * nr + t), v[cols[k * nr + t]], part);
          T acc = v[row] - part;
#pragma unroll
          for (int q = 0; q < 3; ++q)
            if (q < d) acc = fma(-load_as<T, TS>(inn, t * (G - 1) + q), y[q], acc);
          y[d] = acc * load_as<T, TS>(dinv, t);
          v[row] = y[d];
        }
      }
      fence_cta();
      for (int d = 0; d < G; ++d) vf[lrows[gt * G + d]] = static_cast<unsigned char>(phase);
    }
  }
  return true;
}

// Dynamic shared memory of the resident-block Jacobi solve: the slots (one
// block of each kind in mode 2, the largest block in mode 1) and three vectors.
inline size_t jac_slot_a(const Ctx* c, int mode) {
  const size_t a = size_t(mode == 2 ? c->jac_max_bytes[0] : std::max(c->jac_max_bytes[0], c->jac_max_bytes[1]));
  return (a + 127) & ~size_t(127);
}
inline size_t jac_slot_b(const Ctx* c, int mode) {
  return mode == 2 ? (size_t(c->jac_max_bytes[1]) + 127) & ~size_t(127) : 0;
}
inline size_t jac_smem(const Ctx* c, int mode, size_t es) {
  return jac_slot_a(c, mode) + jac_slot_b(c, mode) + 3 * size_t(c->max_m) * es;
}

// Shared memory of the per-row flags (one byte per local row, 16-byte padded).
inline size_t sf_flag_bytes(int max_m) { return (size_t(max_m) + 15) & ~size_t(15); }

template <class T, class TS, int S>
__global__ void __launch_bounds__(kPipeMaxThreads, 1) k_local_sf(const double* __restrict__ r,
                                                           const int* __restrict__ om_ptr,
                                                           const int* __restrict__ om_dofs,
                                                           const int* __restrict__ rec_ptr,
                                                           const uint32_t* __restrict__ rec_off16,
                                                           const uint32_t* __restrict__ rec_bytes,
                                                           const uint8_t* __restrict__ stream, int stage_bytes,
                                                           int vec_bytes, T* __restrict__ zloc,
                                                           const KrylovScalars* __restrict__ ks, int* err,
                                                           long long wait_cycles, int grp, int stall_test,
                                                           int prefetch_bytes, BatchGate gate) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[S];
  __shared__ __align__(8) uint64_t empty[S];
  __shared__ __align__(8) uint64_t gbar;
  __shared__ int s_fail;
  if (ks != nullptr && ks->done) return;
  const int s = blockIdx.x;
  if (gate_sub_off(gate, s)) return;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  const int r0 = rec_ptr[s], nrec = rec_ptr[s + 1] - r0;
  unsigned char* stages = smem_raw;
  unsigned char* vreg = smem_raw + size_t(S) * stage_bytes;
  unsigned char* flags = vreg + vec_bytes;
  const int off = base & 3;
  const int cnt = m > 0 ? (off + m + 3) & ~3 : 0;
  const int m4 = (m + 3) & ~3;
  unsigned char* idx_dst = sizeof(T) == 4 ? vreg : vreg + size_t(4) * m4;
  const int* idx = reinterpret_cast<const int*>(idx_dst) + off;
  T* v = sizeof(T) == 4 ? reinterpret_cast<T*>(vreg) + off : reinterpret_cast<T*>(vreg);
  const int nt = blockDim.x - 32;            // consumer threads
  if (threadIdx.x == 0) {
    for (int j = 0; j < S; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], nt / 32);
    }
    mbar_init(&gbar, 1);
    s_fail = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (int(threadIdx.x) >= nt) {
    pipe_producer<S>(om_dofs, base - off, cnt, idx_dst, &gbar, rec_off16, rec_bytes, r0, nrec, stream, stages,
                     stage_bytes, full, empty, err, wait_cycles, stall_test, prefetch_bytes);
    return;
  }
  volatile int* fail = &s_fail;
  auto set_fail = [&]() {
    if (!*fail) {
      *fail = 1;
      atomicOr(err, 1);
    }
  };
  // ---- consumer warps: indices, gather, flags cleared ----
  {
    const bool ok = m == 0 || mbar_wait_bounded(&gbar, 0, wait_cycles);
    if (consumers_sync_or(!ok, nt)) {
      if (threadIdx.x == 0) atomicOr(err, 1);
      return;
    }
  }
  gather_staged(r, idx, v, m, nt);
  for (int i = threadIdx.x; i < m; i += nt) flags[i] = 0;
  consumers_sync_or(false, nt);
  int phase = 1;
  bool switched = false;          // met the barrier between the sweeps
  for (int i = 0; i < nrec; ++i) {
    const int st = i % S;
    bool ok = !*fail && mbar_wait_bounded(&full[st], (i / S) & 1, wait_cycles);
    if (!ok) set_fail();
    if (ok) {
      const unsigned char* rec = stages + size_t(st) * stage_bytes;
      const int count = reinterpret_cast<const int*>(rec)[7];
      for (int q = 0; q < count && ok; ++q) {
        const unsigned char* next = rec + reinterpret_cast<const int*>(rec)[6];
        if ((reinterpret_cast<const int*>(rec)[5] & kRecUpper) && !switched) {
          consumers_sync(nt);              // the L sweep is complete
          switched = true;
          phase = 2;
        }
        ok = sf_record<T, TS>(rec, v, flags, phase, nt, grp, wait_cycles, fail);
        if (!ok) set_fail();
        rec = next;
      }
    }
    // the warp releases the stage once all its lanes are done with it (never
    // after a failure: the producer then stops on its own bounded wait)
    const bool warp_ok = __all_sync(0xffffffffu, ok);
    if (warp_ok && (threadIdx.x & 31) == 0 && i + S < nrec) mbar_arrive(&empty[st]);
  }
  if (!switched) consumers_sync(nt);
  consumers_sync(nt);
  if (*fail) return;
  for (int i = threadIdx.x; i < m; i += nt) zloc[base + i] = v[i];
}

// ---- Jacobi sweeps on resident blocks (Sec. V-B3, FastSpTRSV) ----
//
// Persistent CTAs (one per SM) take subdomains blockIdx.x, + gridDim.x, ...
// For each, r_s is gathered into shared memory, its L block (one bulk copy
// into slot A, see the setup) is swept from y0 = D^-1 r_s, then its U block
// from the L result, and z_s is written out.  Mode 2: U_s arrives in slot B
// while L_s is swept, and the next subdomain's L block in A while U_s is swept,
// so every factor byte is read from HBM once per apply and its copy overlaps
// the sweeps.  Mode 1 (two blocks do not fit): one slot takes L_s, U_s, the
// next L in turn.  Each sweep updates every row from the previous iterate in
// the order of the unpipelined Jacobi kernel, so the results are the same.
// Every wait is bounded; a wait that runs out sets err[0], and the copies in
// flight land before the CTA returns.

// `sweeps` Jacobi sweeps on T y = rhs with the block in shared memory:
// y0 = D^-1 rhs, y_{k+1} = D^-1 (rhs - (T - D) y_k); returns the buffer
// holding the result (y0 or y1).
template <class T, class TS>
__device__ __forceinline__ T* jac_block_sweeps(const unsigned char* blk, const T* rhs, T* y0, T* y1, int sweeps) {
  const int4 hdr = *reinterpret_cast<const int4*>(blk);
  const int m = hdr.x, K = hdr.y;
  const TS* dinv = reinterpret_cast<const TS*>(blk + 16);
  const TS* vals = reinterpret_cast<const TS*>(blk + hdr.z);
  const uint16_t* cols = reinterpret_cast<const uint16_t*>(blk + hdr.w);
  const int nt = blockDim.x;
  for (int i = threadIdx.x; i < m; i += nt) y0[i] = rhs[i] * load_as<T, TS>(dinv, i);
  __syncthreads();
  T* yo = y0;
  T* yn = y1;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int i = threadIdx.x; i < m; i += nt) {
      T acc = rhs[i];
      for (int k = 0; k < K; ++k) acc -= load_as<T, TS>(vals, k * m + i) * yo[cols[k * m + i]];
      yn[i] = acc * load_as<T, TS>(dinv, i);
    }
    __syncthreads();
    T* t = yo;
    yo = yn;
    yn = t;
  }
  return yo;
}

template <class T, class TS, int MODE>
__global__ void __launch_bounds__(1024, 1) k_local_jac(const double* __restrict__ r,
                                                      const int* __restrict__ om_ptr,
                                                      const int* __restrict__ om_dofs,
                                                      const uint8_t* __restrict__ stream,
                                                      const uint32_t* __restrict__ off16,
                                                      const uint32_t* __restrict__ bytes, int slot_a, int slot_b,
                                                      int max_m, int nsub, int sweeps, T* __restrict__ zloc,
                                                      const KrylovScalars* __restrict__ ks, int* err,
                                                      long long wait_cycles, BatchGate gate, int stall_test) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  if (ks != nullptr && ks->done) return;
  // slot_a, slot_b: the slots' sizes in bytes (slot_b 0 in mode 1)
  unsigned char* slot[2] = {smem_raw, MODE == 2 ? smem_raw + slot_a : smem_raw};
  T* buf0 = reinterpret_cast<T*>(smem_raw + slot_a + slot_b);
  T* buf1 = buf0 + max_m;
  T* buf2 = buf1 + max_m;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int su = MODE == 2 ? 1 : 0;            // slot of the U blocks
  unsigned ph[2] = {0, 0};                     // parity of the next completion of each slot
  bool pending[2] = {false, false};            // thread 0: a copy into the slot is in flight
  auto issue = [&](int sl, int q, int side) {  // thread 0
    const uint32_t nb = bytes[2 * q + side];
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[sl], nb);
    bulk_g2s(slot[sl], stream + size_t(off16[2 * q + side]) * 16, nb, &bar[sl]);
    pending[sl] = true;
  };
  auto live = [&](int q) {                     // the next subdomain at or after q that is not gated off
    while (q < nsub && gate_sub_off(gate, q)) q += gridDim.x;
    return q;
  };
  int s = live(blockIdx.x);
  if (threadIdx.x == 0 && s < nsub) {
    // (failure test: CTA 0's first copy is never issued, so its wait runs out)
    if (!(stall_test && blockIdx.x == 0)) issue(0, s, 0);
    if (MODE == 2) issue(1, s, 1);
  }
  bool failed = false;
  while (s < nsub) {
    const int nx = live(s + int(gridDim.x));
    const int base = om_ptr[s], m = om_ptr[s + 1] - base;
    gather_sub(r, om_dofs, base, m, buf0, threadIdx.x, blockDim.x);
    bool ok = mbar_wait_bounded(&bar[0], ph[0], wait_cycles);
    ph[0] ^= 1u;
    if (threadIdx.x == 0 && ok) pending[0] = false;
    if (__syncthreads_or(!ok)) { failed = true; break; }
    T* yl = jac_block_sweeps<T, TS>(slot[0], buf0, buf1, buf2, sweeps);
    // (the sweeps end with a barrier: slot A is free for its next block)
    if (threadIdx.x == 0) {
      if (MODE == 2) { if (nx < nsub) issue(0, nx, 0); }
      else issue(0, s, 1);
    }
    ok = mbar_wait_bounded(&bar[su], ph[su], wait_cycles);
    ph[su] ^= 1u;
    if (threadIdx.x == 0 && ok) pending[su] = false;
    if (__syncthreads_or(!ok)) { failed = true; break; }
    T* other = yl == buf1 ? buf2 : buf1;
    const T* yu = jac_block_sweeps<T, TS>(slot[su], yl, buf0, other, sweeps);
    for (int i = threadIdx.x; i < m; i += blockDim.x) zloc[base + i] = yu[i];
    __syncthreads();                            // every read of the slot and buffers done
    if (threadIdx.x == 0 && nx < nsub) {
      if (MODE == 2) issue(1, nx, 1);
      else issue(0, nx, 0);
    }
    s = nx;
  }
  if (threadIdx.x == 0) {
    if (failed) atomicOr(err, 1);
    // copies still in flight land before the shared memory goes away (waited
    // for with at least the default bound)
    const long long drain = wait_cycles > kDefaultWaitCycles ? wait_cycles : kDefaultWaitCycles;
    for (int sl = 0; sl < 2; ++sl)
      if (pending[sl]) mbar_wait_bounded(&bar[sl], ph[sl], drain);
  }
}

// One row of a dense inverse times r_s (in shared memory) by a warp: eight
// independent partial sums per lane, so eight loads of the row are in flight
// at once, added in a fixed tree order at the end.
template <class T>
__device__ __forceinline__ T dense_row_dot(const T* __restrict__ Ai, const T* rs, int m, int lane) {
  T acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = T(0);
  int j = lane;
  for (; j + 7 * 32 < m; j += 8 * 32) {
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = Ai[j + 32 * u];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = fma(a[u], rs[j + 32 * u], acc[u]);
  }
  for (int u = 0; j < m; j += 32, ++u) acc[u & 7] = fma(Ai[j], rs[j], acc[u & 7]);
  const T t = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  return warp_sum(t);
}

// Rows of one subdomain per CTA of the dense local solve: one per warp, so a
// row's loads are the only chain a warp waits on (more CTAs each gather r_s).
constexpr int kDenseRows = 8;

// Four consecutive rows of a dense inverse times r_s (in shared memory) by a
// warp: one partial sum per row and lane, each r_s value read once for the
// four rows (two columns per trip, eight loads of the rows in flight), then a
// transposing butterfly: after the exchanges at distance 16 and 8 each lane
// keeps one row's sums, and three more leave row q's total in lanes 8q..8q+7
// -- six additions for the four rows where a shuffle tree per row takes five
// each (FP64 additions issue at the FMA rate).  Rows from nr on are not read.
template <class T>
__device__ __forceinline__ T dense_rows4_dot(const T* __restrict__ A, const T* rs, int m, int nr, int lane) {
  T acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = T(0);
  int j = lane;
  for (; j + 32 < m; j += 64) {
    const T x0 = rs[j], x1 = rs[j + 32];
    T a[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = q < nr ? A[int64_t(q) * m + j] : T(0);
      a[4 + q] = q < nr ? A[int64_t(q) * m + j + 32] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(a[q], x0, acc[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(a[4 + q], x1, acc[q]);
  }
  if (j < m) {
    const T x0 = rs[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(q < nr ? A[int64_t(q) * m + j] : T(0), x0, acc[q]);
  }
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  T b = h16 ? acc[2] : acc[0];
  T e = h16 ? acc[3] : acc[1];
  b += __shfl_xor_sync(0xffffffffu, h16 ? acc[0] : acc[2], 16);
  e += __shfl_xor_sync(0xffffffffu, h16 ? acc[1] : acc[3], 16);
  T f = h8 ? e : b;
  f += __shfl_xor_sync(0xffffffffu, h8 ? b : e, 8);
  f += __shfl_xor_sync(0xffffffffu, f, 4);
  f += __shfl_xor_sync(0xffffffffu, f, 2);
  f += __shfl_xor_sync(0xffffffffu, f, 1);
  return f;
}

// Rows of one subdomain per CTA of the dense local solve: four warps of four
// rows each.
constexpr int kDenseCtaRows = 16;

// Exact local solver: z_s = A_s^-1 r_s with the stored dense inverse
// (symmetric, so row i is read contiguously).  Grid (row chunks of 16, nsub).
template <class T>
__global__ void __launch_bounds__(128) k_local_dense(const double* __restrict__ r,
                                                     const int* __restrict__ om_ptr,
                                                     const int* __restrict__ om_dofs,
                                                     const T* __restrict__ ainv,
                                                     const int64_t* __restrict__ ainv_off,
                                                     T* __restrict__ zloc,
                                                     const KrylovScalars* __restrict__ ks, BatchGate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (ks != nullptr && ks->done) return;
  T* rs = reinterpret_cast<T*>(smem_raw);
  const int s = blockIdx.y;
  if (gate_sub_off(gate, s)) return;
  const int base = om_ptr[s], m = om_ptr[s + 1] - base;
  const int row0 = blockIdx.x * kDenseCtaRows;
  if (row0 >= m) return;
  gather_sub(r, om_dofs, base, m, rs, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = row0 + 4 * w;
  if (i >= m) return;
  const int nr = min(4, m - i);
  const T v = dense_rows4_dot(ainv + ainv_off[s] + int64_t(i) * m, rs, m, nr, lane);
  if ((lane & 7) == 0 && (lane >> 3) < nr) zloc[base + i + (lane >> 3)] = v;
}

// Partial products Phi_b^T r_b.  The first n_cta chunks (more than 256 rows,
// at most 1024, of a block) take one CTA each: the chunk's r is staged in
// shared memory, then each warp takes whole columns, which are contiguous in
// the column-major panel, or (WIDE, for handles whose blocks are wide) the
// warps split the rows and take eight columns at a time.  The small chunks
// (interface components) take one warp each, eight per CTA, with shuffle
// sums; their CTAs are placed first in the grid.
template <class T>
__device__ __forceinline__ void phiT_warp_chunk(int q, const double* __restrict__ r,
                                                const int* __restrict__ brow_ptr,
                                                const int* __restrict__ brow_dof,
                                                const int* __restrict__ bcol_ptr,
                                                const int64_t* __restrict__ phi_off,
                                                const T* __restrict__ phi,
                                                const int* __restrict__ chunk_blk,
                                                const int* __restrict__ chunk_r0,
                                                const int* __restrict__ chunk_r1,
                                                const int* __restrict__ chunk_slot,
                                                double* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int b = chunk_blk[q];
  const int p0 = brow_ptr[b], nr = brow_ptr[b + 1] - p0;
  const int i0 = chunk_r0[q], i1 = chunk_r1[q];
  const int k = bcol_ptr[b + 1] - bcol_ptr[b];
  const T* Ph = phi + phi_off[b];
  for (int c0 = 0; c0 < k; c0 += 8) {
    const int kc = min(8, k - c0);
    T acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = T(0);
    // four rows per lane and trip: indices, then values, then the products
    for (int ib = i0 + lane; ib < i1; ib += 4 * 32) {
      int g[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) g[j] = ib + 32 * j < i1 ? brow_dof[p0 + ib + 32 * j] : -1;
      uint64_t rb[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) rb[j] = g[j] >= 0 ? load_bits(r, g[j]) : 0ull;
      T rv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) rv[j] = narrow_bits<T>(rb[j]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (g[j] < 0) continue;
        const T* col = Ph + int64_t(c0) * nr + ib + 32 * j;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < kc) acc[u] = fma(col[int64_t(u) * nr], rv[j], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u < kc) {
        const T t = warp_sum(acc[u]);
        if (lane == 0) partial[chunk_slot[q] + c0 + u] = double(t);
      }
    }
  }
}

// Sums of eight values over a warp's lanes, transposed: the exchanges at
// distance 16, 8 and 4 each halve the values a lane keeps (4 + 2 + 1
// additions), two more complete the sums, and lanes 4q..4q+3 return the sum of
// value q.
template <class T>
__device__ __forceinline__ T phiT_butterfly8(const T (&v)[8], int lane) {
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0;
  T a[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T keep = h16 ? v[4 + j] : v[j], give = h16 ? v[j] : v[4 + j];
    a[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
  }
  T c[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T keep = h8 ? a[2 + j] : a[j], give = h8 ? a[j] : a[2 + j];
    c[j] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
  }
  T e = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 4);
  e += __shfl_xor_sync(0xffffffffu, e, 2);
  e += __shfl_xor_sync(0xffffffffu, e, 1);
  return e;
}

template <class T, bool WIDE>
__global__ void __launch_bounds__(256, WIDE || sizeof(T) == 8 ? 4 : 6) k_phiT(int n_chunks, int n_cta, const double* __restrict__ r,
                                              const int* __restrict__ brow_ptr,
                                              const int* __restrict__ brow_dof,
                                              const int* __restrict__ bcol_ptr,
                                              const int64_t* __restrict__ phi_off,
                                              const T* __restrict__ phi,
                                              const int* __restrict__ chunk_blk,
                                              const int* __restrict__ chunk_r0,
                                              const int* __restrict__ chunk_r1,
                                              const int* __restrict__ chunk_slot,
                                              double* __restrict__ partial,
                                              const KrylovScalars* __restrict__ ks, BatchGate gate) {
  __shared__ T rs[kPhiChunkRows];          // r of a chunk
  __shared__ T red[WIDE ? 8 : 1][8];       // the warps' sums of eight columns
  if (ks != nullptr && ks->done) return;
  // the small chunks' CTAs come first in the grid, so that their longer
  // chains of dependent loads overlap the big chunks instead of trailing them
  const int n_warp_ctas = (n_chunks - n_cta + 7) / 8;
  if (int(blockIdx.x) < n_warp_ctas) {
    // warp path: no CTA-wide barrier below
    const int q = n_cta + int(blockIdx.x) * 8 + (threadIdx.x >> 5);
    if (q < n_chunks && !gate_blk_off(gate, chunk_blk[q]))
      phiT_warp_chunk<T>(q, r, brow_ptr, brow_dof, bcol_ptr, phi_off, phi, chunk_blk, chunk_r0, chunk_r1,
                         chunk_slot, partial);
    return;
  }
  const int q = int(blockIdx.x) - n_warp_ctas;
  const int b = chunk_blk[q];
  if (gate_blk_off(gate, b)) return;
  const int p0 = brow_ptr[b], nr = brow_ptr[b + 1] - p0;
  const int i0 = chunk_r0[q], rows = chunk_r1[q] - i0;
  const int k = bcol_ptr[b + 1] - bcol_ptr[b];
  // r of the chunk's rows into shared memory (four rows per thread in flight)
  for (int ib = threadIdx.x; ib < rows; ib += 4 * 256) {
    int g[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) g[j] = ib + 256 * j < rows ? brow_dof[p0 + i0 + ib + 256 * j] : -1;
    uint64_t rb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) rb[j] = g[j] >= 0 ? load_bits(r, g[j]) : 0ull;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (g[j] >= 0) rs[ib + 256 * j] = narrow_bits<T>(rb[j]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if constexpr (WIDE) {
    // eight columns at a time: warp w takes rows w * 32 + lane + 256 j, two
    // rows per trip with the eight columns' values of both loaded together
    // (sixteen coalesced loads in flight per lane, r read once per row); then
    // a transposing butterfly leaves column q's warp sum in lanes 4q..4q+3 and
    // the eight warps' sums are added in warp order
    const T* P0 = phi + phi_off[b] + i0;
    for (int c0 = 0; c0 < k; c0 += 8) {
      const int kc = min(8, k - c0);
      T acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = T(0);
      for (int i = w * 32 + lane; i < rows; i += 512) {
        const bool two = i + 256 < rows;
        const T x0 = rs[i], x1 = two ? rs[i + 256] : T(0);
        T a0[8], a1[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const T* col = P0 + int64_t(c0 + u) * nr;
          a0[u] = u < kc ? col[i] : T(0);
          a1[u] = u < kc && two ? col[i + 256] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fma(a1[u], x1, fma(a0[u], x0, acc[u]));
      }
      const T v = phiT_butterfly8(acc, lane);
      if ((lane & 3) == 0) red[w][lane >> 2] = v;
      __syncthreads();
      if (threadIdx.x < kc) {
        T t = red[0][threadIdx.x];
#pragma unroll
        for (int ww = 1; ww < 8; ++ww) t += red[ww][threadIdx.x];
        partial[chunk_slot[q] + c0 + threadIdx.x] = double(t);
      }
      __syncthreads();
    }
  } else {
    // one warp per column: the column is contiguous in the block's panel
    for (int u = w; u < k; u += 8) {
      const T* col = phi + phi_off[b] + int64_t(u) * nr + i0;
      T acc[4] = {T(0), T(0), T(0), T(0)};
      int i = lane;
      // software-pipelined: the next four values of the column are loaded
      // before the current four are used
      if (i + 96 < rows) {
        T cv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cv[j] = col[i + 32 * j];
        for (; i + 128 + 96 < rows; i += 128) {
          T nx[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) nx[j] = col[i + 128 + 32 * j];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = fma(cv[j], rs[i + 32 * j], acc[j]);
#pragma unroll
          for (int j = 0; j < 4; ++j) cv[j] = nx[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fma(cv[j], rs[i + 32 * j], acc[j]);
        i += 128;
      }
      for (; i < rows; i += 32) acc[0] = fma(col[i], rs[i], acc[0]);
      const T t = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
      if (lane == 0) partial[chunk_slot[q] + u] = double(t);
    }
  }
}

__global__ void k_coarse_c(int n0, const int* __restrict__ cs_ptr, const int* __restrict__ cs_idx,
                           const double* __restrict__ partial, double* __restrict__ c,
                           float* __restrict__ c32, const KrylovScalars* __restrict__ ks, BatchGate gate) {
  if (ks != nullptr && ks->done) return;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n0; l += gridDim.x * blockDim.x) {
    if (gate_col_off(gate, l)) continue;
    double v = 0.0;
    for (int q = cs_ptr[l]; q < cs_ptr[l + 1]; ++q) v += partial[cs_idx[q]];
    c[l] = v;
    if (c32 != nullptr) c32[l] = float(v);
  }
}

// y = A0^-1 c with the explicit inverse (one dense block per problem), in the
// inverse's stored type TA (FP64, or FP32 for a single-precision apply, whose
// FMAs then leave B300's slow FP64 pipe).  Two warps per row, each over half
// of the columns with eight independent FMA chains per lane; the halves are
// added in a fixed order.  c is read through L1/L2, not staged in shared
// memory, so the CTAs need almost none and fit beside the local solve's CTAs
// on the same SMs (the two branches of the apply overlap).
template <class TA>
__global__ void __launch_bounds__(256) k_coarse_gemv(int n0, const TA* __restrict__ Ainv,
                                                     const int* __restrict__ coarse_prob,
                                                     const int* __restrict__ prob_c0,
                                                     const int64_t* __restrict__ a0_off,
                                                     const TA* __restrict__ c,
                                                     double* __restrict__ y, float* __restrict__ y32,
                                                     const KrylovScalars* __restrict__ ks, BatchGate gate) {
  __shared__ TA half_sum[4][2];
  if (ks != nullptr && ks->done) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int slot = w >> 1, h = w & 1;                  // row slot in the CTA, half of the row
  for (int row0 = blockIdx.x * 4; row0 < n0; row0 += gridDim.x * 4) {
    const int row = row0 + slot;
    TA acc = TA(0);
    const bool live = row < n0 && !gate_col_off(gate, row);
    if (live) {
      const int pr = coarse_prob[row];
      const int cp = prob_c0[pr], np = prob_c0[pr + 1] - cp;
      const TA* Ar = Ainv + a0_off[pr] + int64_t(row - cp) * np;
      const TA* cv = c + cp;
      // short rows (small problems of a batch) go whole to the first warp
      const int split = np >= 1024 ? np / 2 : np;
      const int j0 = h == 0 ? 0 : split, j1 = h == 0 ? split : np;
      TA a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = TA(0);
      int j = j0 + lane;
      // software-pipelined: the next eight values of the row are loaded before
      // the current eight are used, so two trips' loads are in flight
      if (j + 7 * 32 < j1) {
        TA m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) m[u] = Ar[j + 32 * u];
        for (; j + 15 * 32 < j1; j += 8 * 32) {
          TA nx[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) nx[u] = Ar[j + 8 * 32 + 32 * u];
#pragma unroll
          for (int u = 0; u < 8; ++u) a[u] = fma(m[u], cv[j + 32 * u], a[u]);
#pragma unroll
          for (int u = 0; u < 8; ++u) m[u] = nx[u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(m[u], cv[j + 32 * u], a[u]);
        j += 8 * 32;
      }
      for (; j < j1; j += 32) a[0] = fma(Ar[j], cv[j], a[0]);
      acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
      acc = warp_sum(acc);
    }
    if (lane == 0) half_sum[slot][h] = acc;
    __syncthreads();
    if (h == 0 && lane == 0 && live) {
      const TA v = half_sum[slot][0] + half_sum[slot][1];
      y[row] = double(v);
      if (y32 != nullptr) y32[row] = float(v);   // converted once, not per scatter position
    }
    __syncthreads();
  }
}

// yb[i] = y[bcol[i]]: the coarse solution at every column slot of the Phi
// blocks, in the apply's precision, so the scatter-add reads one array (no
// column index, then value, per Phi entry).
template <class T>
__global__ void k_coarse_slots(int nslots, const int* __restrict__ bcol, const T* __restrict__ y,
                               T* __restrict__ yb, const KrylovScalars* __restrict__ ks) {
  if (ks != nullptr && ks->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += gridDim.x * blockDim.x) yb[i] = y[bcol[i]];
}

// u_p = (Phi y) at block-row position p, in the preconditioner's precision T,
// eight Phi columns in flight per thread (each sum in column order), y read
// through the block-column map `bcol` (the values the column-slot gather
// copies, so the sums are the same), or with bcol null from the slots `y`
// themselves (wide blocks, whose many map reads per position cost more than
// the gather).  It runs on the coarse stream after the GEMV, beside the local
// solves, so the scatter-add only adds u; positions of stopped problems are
// skipped.
template <class T>
__global__ void __launch_bounds__(256) k_prolong(int n, const int* __restrict__ pos_blk,
                                                 const int* __restrict__ brow_ptr,
                                                 const int* __restrict__ bcol_ptr,
                                                 const int64_t* __restrict__ phi_off, const T* __restrict__ phi,
                                                 const int* __restrict__ bcol, const T* __restrict__ y,
                                                 T* __restrict__ ub, const KrylovScalars* __restrict__ ks,
                                                 BatchGate gate) {
  if (ks != nullptr && ks->done) return;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int b = pos_blk[p];
    if (gate_blk_off(gate, b)) continue;
    const int c0 = bcol_ptr[b], k = bcol_ptr[b + 1] - c0, p0 = brow_ptr[b], nr = brow_ptr[b + 1] - p0;
    T acc = T(0);
    if (k > 0) {
      const T* ph = phi + phi_off[b] + (p - p0);
      int u = 0;
      for (; u + 8 <= k; u += 8) {
        T pv[8], yv[8];
        int cj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          pv[q] = ph[int64_t(u + q) * nr];
          cj[q] = bcol != nullptr ? bcol[c0 + u + q] : c0 + u + q;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) yv[q] = y[cj[q]];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc = fma(pv[q], yv[q], acc);
      }
      for (; u < k; ++u) acc = fma(ph[int64_t(u) * nr], y[bcol != nullptr ? bcol[c0 + u] : c0 + u], acc);
    }
    ub[p] = acc;
  }
}

// z_g = sum over subdomains containing g of (z_s)_g (ascending subdomain
// order) + (Phi y)_g (formed here, or with PROL read from k_prolong's output
// by position), one unknown per thread over the block-row positions
// (pos_blk gives the Phi block of each position), summed in the
// preconditioner's precision T and widened once.  With `dots`, also
// (r, z_new) and (r, z_old), reduced by the last CTA, which sets beta and
// (r, z) for the PCG update.
//
// Each thread takes NP positions per trip and moves through them in phases,
// so that the loads of a phase are in flight together for all of them:
// indices; then r, the first two pulls and the block's shape; then the local
// values and the Phi row, four columns at a time (each position's sum is still
// formed in the order pulls, then Phi columns).
template <class T, int NP, int CB, bool PROL>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (CB > 4 ? 3 : 5) : (CB > 4 ? 2 : 3)) k_combine(
    int n, const double* __restrict__ r, double* __restrict__ z, const int* __restrict__ brow_dof,
    const int* __restrict__ pos_blk, const int* __restrict__ brow_ptr,
    const int* __restrict__ bcol_ptr, const int64_t* __restrict__ phi_off, const T* __restrict__ phi,
    const T* __restrict__ yb, const T* __restrict__ ub, const int* __restrict__ pull_ptr,
    const int* __restrict__ pull_pos,
    const T* __restrict__ zloc, int dots, double* __restrict__ red, KrylovScalars* ks, BatchGate gate) {
  __shared__ double sh[32];
  if (ks != nullptr && ks->done) return;
  double d_new = 0.0, d_old = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += NP * stride) {
    int g[NP], b[NP], q0[NP], q1[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int pj = p + j * stride;
      const bool in = pj < n;
      b[j] = in ? pos_blk[pj] : 0;
      g[j] = in ? brow_dof[pj] : -1;
      q0[j] = in ? pull_ptr[pj] : 0;
      q1[j] = in ? pull_ptr[pj + 1] : 0;
    }
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (g[j] >= 0 && gate_blk_off(gate, b[j])) g[j] = -1;
    double rg[NP], zo[NP];
    int pull0[NP], pull1[NP], c0[NP], k[NP], p0[NP], nr[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const bool live = g[j] >= 0;
      rg[j] = live && dots ? r[g[j]] : 0.0;
      zo[j] = live && dots > 1 ? z[g[j]] : 0.0;
      pull0[j] = live && q0[j] < q1[j] ? pull_pos[q0[j]] : -1;
      pull1[j] = live && q0[j] + 1 < q1[j] ? pull_pos[q0[j] + 1] : -1;
      c0[j] = live ? bcol_ptr[b[j]] : 0;
      k[j] = live ? bcol_ptr[b[j] + 1] - c0[j] : 0;
      p0[j] = live ? brow_ptr[b[j]] : 0;
      nr[j] = live ? brow_ptr[b[j] + 1] - p0[j] : 0;
    }
    T acc[NP];
    const T* ph[NP];
    int kmax = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      acc[j] = T(0);
      if (pull0[j] >= 0) acc[j] += zloc[pull0[j]];
      if (pull1[j] >= 0) acc[j] += zloc[pull1[j]];
      for (int q = q0[j] + 2; q < q1[j]; ++q) acc[j] += zloc[pull_pos[q]];
      ph[j] = phi + (k[j] > 0 ? phi_off[b[j]] + (p + j * stride - p0[j]) : 0);
      kmax = max(kmax, k[j]);
    }
    if constexpr (PROL) {
      // Phi y formed beside the local solves (k_prolong), one value per position
#pragma unroll
      for (int j = 0; j < NP; ++j)
        if (g[j] >= 0) acc[j] += ub[p + j * stride];
      kmax = 0;
    }
    for (int u0 = 0; u0 < kmax; u0 += CB) {
      T pv[NP][CB], yv[NP][CB];
#pragma unroll
      for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int u = 0; u < CB; ++u) {
          const bool on = u0 + u < k[j];
          pv[j][u] = on ? ph[j][int64_t(u0 + u) * nr[j]] : T(0);
          yv[j][u] = on ? yb[c0[j] + u0 + u] : T(0);
        }
#pragma unroll
      for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int u = 0; u < CB; ++u)
          if (u0 + u < k[j]) acc[j] = fma(pv[j][u], yv[j][u], acc[j]);
    }
    double a[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) a[j] = widen<T>(acc[j]);
    if (dots) {
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        if (g[j] < 0) continue;
        if (dots > 1) d_old = fma(rg[j], zo[j], d_old);
        d_new = fma(rg[j], a[j], d_new);
      }
    }
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (g[j] >= 0) z[g[j]] = a[j];
  }
  if (!dots) return;
  const double tn = block_sum(d_new, sh);
  const double to = block_sum(d_old, sh);
  if (threadIdx.x == 0) {
    red[2 * blockIdx.x] = tn;
    red[2 * blockIdx.x + 1] = to;
  }
  if (arrive_last(&ks->ticket[2])) {
    double sn = 0.0, so = 0.0;
    for (int q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
      sn += __ldcg(red + 2 * q);
      so += __ldcg(red + 2 * q + 1);
    }
    sn = block_sum(sn, sh);
    so = block_sum(so, sh);
    if (threadIdx.x == 0) {
      const double num = dots > 1 ? (sn - so) : sn;
      ks->beta = num / ks->rz;
      ks->rz_oldz = so;
      ks->rz_new = sn;
      ks->rz = sn;
    }
  }
}

// ---- PCG as one persistent kernel ----
//
// For small problems the PCG iteration is bound by its launches (config 1: ten
// kernels of a few microseconds each), so single-problem handles with dense
// exact local solves and a small coarse space (n0 <= kPersistMaxN0) can run the
// whole loop in one cooperative launch.  Each iteration is the graph body's
// sequence, phase by phase over the whole grid, with a grid barrier (bounded
// spin on a monotonic counter) between phases: q = A p and (p, q); r -= alpha q,
// ||r||^2, x += alpha p, the stopping test; the dense local solves and Phi^T r;
// the coarse solve (every CTA, redundantly, in shared memory) and the
// scatter-add with the PCG dots; p = z + beta p.  Every CTA sums the per-CTA
// partials of a reduction itself in the same fixed order, so all agree on
// alpha, beta and the stopping decision without another barrier.  A barrier
// wait that runs out sets the error flag and the CTA returns (the others' waits
// run out in turn).
constexpr int kPersistMaxN0 = 128;
constexpr int kPersistPerSM = 1;   // CTAs per SM: fewer arrivals on the barrier counter

struct PersistArgs {
  int n, nsub, n0, n_chunks, n_units, dots;
  const int* rowptr; const int* colind; const int16_t* dcol16; const double* val;
  double *x, *r, *p, *q, *z;
  const int* om_ptr; const int* om_dofs; const void* ainv; const int64_t* ainv_off; const int* unit_ptr; void* zloc;
  const int* brow_ptr; const int* brow_dof; const int* bcol_ptr; const int* bcol; const int64_t* phi_off;
  const void* phi; const int* chunk_blk; const int* chunk_r0; const int* chunk_r1; const int* chunk_slot;
  double* partial; const int* cs_ptr; const int* cs_idx; const void* a0inv;
  const int* pos_blk; const int* pull_ptr; const int* pull_pos;
  double* red; unsigned* bar; KrylovScalars* ks; int* err; long long wait_cycles; int max_m;
  int stall_test;   // CTA 0 withholds its first barrier arrival (the failure test)
};

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, long long cycles, int* s_flag,
                                             bool withhold = false) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (!withhold) atomicAdd(bar, 1u);
    const volatile unsigned* vb = bar;
    int ok = 1;
    if (*vb < target) {
      const long long t0 = clock64();
      while (*vb < target) {
        __nanosleep(64);          // fewer polls of the shared line
        if (clock64() - t0 > cycles) { ok = 0; break; }
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// The grid-wide sum of `count` per-CTA partials, in index order, in every thread.
__device__ __forceinline__ double grid_total(const double* part, int count, double* sh, double* s_out) {
  const double v = sum_partials(part, count, sh);
  if (threadIdx.x == 0) *s_out = v;
  __syncthreads();
  const double t = *s_out;
  __syncthreads();
  return t;
}

template <class T>
__global__ void __launch_bounds__(256) k_pcg_persistent(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ double s_out;
  __shared__ int s_flag;
  T* rs = reinterpret_cast<T*>(smem_raw);                                     // r_s of one subdomain
  T* cs = reinterpret_cast<T*>(smem_raw + ((size_t(a.max_m) * sizeof(T) + 15) & ~size_t(15)));
  T* ys = cs + kPersistMaxN0;                                                 // coarse rhs and solution
  KrylovScalars* ks = a.ks;
  const int G = gridDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, stride = G * blockDim.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * (blockDim.x >> 5) + w, nwarps = G * (blockDim.x >> 5);
  double rz = ks->rz;
  int iter = ks->iter;
  const int maxit = ks->maxit;
  const double tol2 = ks->tol2;
  unsigned epoch = 0;
  double* red0 = a.red;            // (p, q)
  double* red1 = a.red + G;        // ||r||^2
  double* red2 = a.red + 2 * G;    // the scatter-add's two dots
  const T* ainv = static_cast<const T*>(a.ainv);
  const T* phi = static_cast<const T*>(a.phi);
  const T* a0 = static_cast<const T*>(a.a0inv);
  T* zloc = static_cast<T*>(a.zloc);
  for (;;) {
    // q = A p, (p, q)
    double dot = 0.0;
    for (int row = gtid; row < a.n; row += stride) {
      const int e0 = a.rowptr[row], e1 = a.rowptr[row + 1];
      double acc = 0.0;
      for (int e = e0; e < e1; ++e) {
        const int col = a.dcol16 != nullptr ? row + a.dcol16[e] : a.colind[e];
        acc = fma(a.val[e], a.p[col], acc);
      }
      a.q[row] = acc;
      dot = fma(a.p[row], acc, dot);
    }
    {
      const double t = block_sum(dot, sh);
      if (threadIdx.x == 0) red0[blockIdx.x] = t;
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.wait_cycles, &s_flag, a.stall_test && blockIdx.x == 0 && epoch == 1))
      break;
    const double pq = grid_total(red0, G, sh, &s_out);
    const double alpha = rz / pq;
    // r -= alpha q, ||r||^2, x += alpha p
    double rr = 0.0;
    for (int i = gtid; i < a.n; i += stride) {
      const double ri = fma(-alpha, a.q[i], a.r[i]);
      a.r[i] = ri;
      rr = fma(ri, ri, rr);
      a.x[i] = fma(alpha, a.p[i], a.x[i]);
    }
    {
      const double t = block_sum(rr, sh);
      if (threadIdx.x == 0) red1[blockIdx.x] = t;
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.wait_cycles, &s_flag)) break;
    rr = grid_total(red1, G, sh, &s_out);
    ++iter;
    int done = 0, bad = 0;
    if (!isfinite(rr) || !isfinite(alpha) || !(pq > 0.0)) { bad = 1; done = 1; }
    else if (rr <= tol2) done = 1;
    else if (iter >= maxit) done = 1;
    if (done) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        ks->rr = rr; ks->pq = pq; ks->alpha = alpha; ks->iter = iter; ks->bad = bad; ks->done = 1; ks->rz = rz;
      }
      return;
    }
    // dense local solves, kDenseRows rows of one subdomain per unit
    for (int u = blockIdx.x; u < a.n_units; u += G) {
      int lo = 0, hi = a.nsub;                  // the subdomain of unit u
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.unit_ptr[mid] <= u) lo = mid; else hi = mid;
      }
      const int s = lo;
      const int base = a.om_ptr[s], m = a.om_ptr[s + 1] - base;
      const int row0 = (u - a.unit_ptr[s]) * kDenseRows;
      gather_sub(a.r, a.om_dofs, base, m, rs, threadIdx.x, blockDim.x);
      __syncthreads();
      const T* A = ainv + a.ainv_off[s];
      for (int rw = w; rw < kDenseRows; rw += 8) {
        const int i = row0 + rw;
        if (i >= m) break;
        const T acc = dense_row_dot(A + int64_t(i) * m, rs, m, lane);
        if (lane == 0) zloc[base + i] = acc;
      }
      __syncthreads();
    }
    // Phi^T r by chunks, a warp each
    for (int qq = gwarp; qq < a.n_chunks; qq += nwarps)
      phiT_warp_chunk<T>(qq, a.r, a.brow_ptr, a.brow_dof, a.bcol_ptr, a.phi_off, phi, a.chunk_blk, a.chunk_r0,
                         a.chunk_r1, a.chunk_slot, a.partial);
    if (!grid_barrier(a.bar, (++epoch) * G, a.wait_cycles, &s_flag)) break;
    // coarse solve, redundantly in every CTA: c = Phi^T r by columns, y = A0^-1 c
    for (int l = threadIdx.x; l < a.n0; l += blockDim.x) {
      double v = 0.0;
      for (int qq = a.cs_ptr[l]; qq < a.cs_ptr[l + 1]; ++qq) v += __ldcg(a.partial + a.cs_idx[qq]);
      cs[l] = static_cast<T>(v);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < a.n0; l += blockDim.x) {
      T v = T(0);
      for (int j = 0; j < a.n0; ++j) v = fma(a0[int64_t(l) * a.n0 + j], cs[j], v);
      ys[l] = v;
    }
    __syncthreads();
    // z = sum_s R_s^T z_s + Phi y, (r, z) and (r, z_old)
    double d_new = 0.0, d_old = 0.0;
    for (int pp = gtid; pp < a.n; pp += stride) {
      const int g = a.brow_dof[pp], b = a.pos_blk[pp];
      T acc = T(0);
      for (int q2 = a.pull_ptr[pp]; q2 < a.pull_ptr[pp + 1]; ++q2) acc += zloc[a.pull_pos[q2]];
      const int c0 = a.bcol_ptr[b], k = a.bcol_ptr[b + 1] - c0;
      if (k > 0) {
        const int p0 = a.brow_ptr[b], nr = a.brow_ptr[b + 1] - p0;
        const T* Ph = phi + a.phi_off[b] + (pp - p0);
        for (int u = 0; u < k; ++u) acc = fma(Ph[int64_t(u) * nr], ys[a.bcol[c0 + u]], acc);
      }
      const double zg = widen<T>(acc);
      const double rg = a.r[g];
      if (a.dots > 1) d_old = fma(rg, a.z[g], d_old);
      d_new = fma(rg, zg, d_new);
      a.z[g] = zg;
    }
    {
      const double tn = block_sum(d_new, sh);
      const double to = block_sum(d_old, sh);
      if (threadIdx.x == 0) { red2[2 * blockIdx.x] = tn; red2[2 * blockIdx.x + 1] = to; }
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.wait_cycles, &s_flag)) break;
    double sn = 0.0, so = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
      sn += __ldcg(red2 + 2 * i);
      so += __ldcg(red2 + 2 * i + 1);
    }
    sn = block_sum(sn, sh);
    so = block_sum(so, sh);
    if (threadIdx.x == 0) { s_out = sn; sh[0] = so; }
    __syncthreads();
    sn = s_out;
    so = sh[0];
    __syncthreads();
    const double beta = (a.dots > 1 ? (sn - so) : sn) / rz;
    rz = sn;
    // p = z + beta p
    for (int i = gtid; i < a.n; i += stride) a.p[i] = fma(beta, a.p[i], a.z[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ks->iter = iter; ks->rr = rr; ks->rz = rz; ks->rz_new = sn; ks->rz_oldz = so; ks->beta = beta;
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.wait_cycles, &s_flag)) break;
  }
  if (threadIdx.x == 0) atomicOr(a.err, 1);
}

template <class T>
EllDev<T> ell(const Ctx* c, bool lower) {
  EllDev<T> e;
  if (lower) {
    e.sub_lev = c->L_sub_lev; e.lev = c->L_lev; e.lrows = c->L_lrows; e.col = c->L_col;
    e.val = static_cast<const T*>(c->L_val); e.dinv = static_cast<const T*>(c->L_dinv);
  } else {
    e.sub_lev = c->U_sub_lev; e.lev = c->U_lev; e.lrows = c->U_lrows; e.col = c->U_col;
    e.val = static_cast<const T*>(c->U_val); e.dinv = static_cast<const T*>(c->U_dinv);
  }
  e.grp = c->dpn;
  return e;
}

template <class T>
gdsw_status launch_local(Ctx* c, const double* r, cudaStream_t s, const KrylovScalars* ks, const BatchGate& gate) {
  T* zl = static_cast<T*>(c->zloc);
  if (c->mf) return mf_launch_local(c, r, s, ks);
  if (c->opt.local_solver == GDSW_LOCAL_EXACT) {
    const size_t shm = size_t(c->max_m) * sizeof(T);
    dim3 grid((c->max_m + kDenseCtaRows - 1) / kDenseCtaRows, c->nsub);
    k_local_dense<T><<<grid, 128, shm, s>>>(r, c->om_ptr, c->om_dofs, static_cast<const T*>(c->ainv),
                                            c->ainv_off, zl, ks, gate);
  } else if (c->node_stages > 0) {
    // node programs (FP32, three unknowns per node)
    if constexpr (std::is_same<T, float>::value) {
      const size_t shm = nodes_smem_bytes(c->node_stages, c->node_slot_bytes, c->max_m);
#define GDSW_NODES_LAUNCH(TT, LL)                                                                           \
  k_local_nodes<TT, LL><<<c->nsub, TT, shm, s>>>(r, c->om_ptr, c->om_dofs, c->node_ptr, c->node_piece,        \
                                                c->node_stream, c->node_stages, c->node_slot_bytes, zl, ks,   \
                                                c->derr, c->wait_cycles, c->stall_test, gate)
      const int sel = (c->node_threads == 256 ? 0 : 3) + (c->node_lanes == 2 ? 0 : c->node_lanes == 4 ? 1 : 2);
      switch (sel) {
        case 0: GDSW_NODES_LAUNCH(256, 2); break;
        case 1: GDSW_NODES_LAUNCH(256, 4); break;
        case 2: GDSW_NODES_LAUNCH(256, 8); break;
        case 3: GDSW_NODES_LAUNCH(512, 2); break;
        case 4: GDSW_NODES_LAUNCH(512, 4); break;
        default: GDSW_NODES_LAUNCH(512, 8); break;
      }
#undef GDSW_NODES_LAUNCH
    }
  } else if (c->step_depth > 0) {
    // row programs with per-thread prefetch (FP32, rows of at most 3 entries)
    if constexpr (std::is_same<T, float>::value) {
      const size_t shm = steps_smem_bytes(c->step_depth, c->step_max, c->max_m);
#define GDSW_STEPS_LAUNCH(DD)                                                                                  \
  k_local_steps<DD><<<c->nsub, kStepRows, shm, s>>>(r, c->om_ptr, c->om_dofs, c->step_ptr, c->steps,           \
                                                   reinterpret_cast<const float4*>(c->step_a),                 \
                                                   reinterpret_cast<const uint2*>(c->step_c), c->step_max, zl, \
                                                   ks, gate)
      switch (c->step_depth) {
        case 4: GDSW_STEPS_LAUNCH(4); break;
        case 12: GDSW_STEPS_LAUNCH(12); break;
        default: GDSW_STEPS_LAUNCH(8); break;
      }
#undef GDSW_STEPS_LAUNCH
    }
  } else if (c->rec_stages > 0 && c->rec_sf) {
    // without a barrier per level (one unknown per row group of at most 4, rows of up to 8 entries)
    const int vb = static_cast<int>(pipe_vector_bytes(c->max_m, sizeof(T)));
    const size_t shm = size_t(c->rec_stages) * c->rec_stage_bytes + vb + sf_flag_bytes(c->max_m);
#define GDSW_SF_LAUNCH(TS, SS)                                                                             \
  k_local_sf<T, TS, SS><<<c->nsub, c->rec_consumers + 32, shm, s>>>(                                      \
      r, c->om_ptr, c->om_dofs, c->rec_ptr, c->rec_off16, c->rec_bytes, c->rec_stream, c->rec_stage_bytes, \
      vb, zl, ks, c->derr, c->wait_cycles, c->dpn, c->stall_test, c->rec_prefetch, gate)
    if (c->fp16) {
      if constexpr (std::is_same<T, float>::value) {
        switch (c->rec_stages) {
          case 2: GDSW_SF_LAUNCH(__half, 2); break;
          case 4: GDSW_SF_LAUNCH(__half, 4); break;
          case 8: GDSW_SF_LAUNCH(__half, 8); break;
          default: GDSW_SF_LAUNCH(__half, 16); break;
        }
      }
    } else {
      switch (c->rec_stages) {
        case 2: GDSW_SF_LAUNCH(T, 2); break;
        case 4: GDSW_SF_LAUNCH(T, 4); break;
        case 8: GDSW_SF_LAUNCH(T, 8); break;
        default: GDSW_SF_LAUNCH(T, 16); break;
      }
    }
#undef GDSW_SF_LAUNCH
  } else if (c->rec_stages > 0) {
    const size_t shm = size_t(c->rec_stages) * c->rec_stage_bytes + pipe_vector_bytes(c->max_m, sizeof(T));
    const int key = c->rec_stages * 100 + c->rec_tpr;
    if (c->fp16) {
      if constexpr (std::is_same<T, float>::value) {
#define GDSW_PIPE_LAUNCH(SS, TP)                                                                            \
  k_local_pipe<T, __half, SS, TP><<<c->nsub, c->rec_consumers + 32, shm, s>>>(r, c->om_ptr, c->om_dofs, c->rec_ptr,            \
                                                            c->rec_off16, c->rec_bytes, c->rec_stream,       \
                                                            c->rec_stage_bytes, zl, ks, c->derr,             \
                                                            c->wait_cycles, c->dpn, c->stall_test,           \
                                                            c->rec_prefetch, gate)
        switch (key) {
          case 201: GDSW_PIPE_LAUNCH(2, 1); break;
          case 401: GDSW_PIPE_LAUNCH(4, 1); break;
          case 801: GDSW_PIPE_LAUNCH(8, 1); break;
          case 1601: GDSW_PIPE_LAUNCH(16, 1); break;
          case 208: GDSW_PIPE_LAUNCH(2, 8); break;
          case 408: GDSW_PIPE_LAUNCH(4, 8); break;
          case 808: GDSW_PIPE_LAUNCH(8, 8); break;
          default: GDSW_PIPE_LAUNCH(16, 8); break;
        }
#undef GDSW_PIPE_LAUNCH
      }
    } else {
#define GDSW_PIPE_LAUNCH(SS, TP)                                                                     \
  k_local_pipe<T, T, SS, TP><<<c->nsub, c->rec_consumers + 32, shm, s>>>(r, c->om_ptr, c->om_dofs, c->rec_ptr, c->rec_off16, \
                                                       c->rec_bytes, c->rec_stream, c->rec_stage_bytes, zl, \
                                                       ks, c->derr, c->wait_cycles, c->dpn, c->stall_test,  \
                                                       c->rec_prefetch, gate)
      switch (key) {
        case 201: GDSW_PIPE_LAUNCH(2, 1); break;
        case 401: GDSW_PIPE_LAUNCH(4, 1); break;
        case 801: GDSW_PIPE_LAUNCH(8, 1); break;
        case 1601: GDSW_PIPE_LAUNCH(16, 1); break;
        case 208: GDSW_PIPE_LAUNCH(2, 8); break;
        case 408: GDSW_PIPE_LAUNCH(4, 8); break;
        case 808: GDSW_PIPE_LAUNCH(8, 8); break;
        default: GDSW_PIPE_LAUNCH(16, 8); break;
      }
    }
#undef GDSW_PIPE_LAUNCH
  } else if (c->jac_mode > 0) {
    const size_t shm = jac_smem(c, c->jac_mode, sizeof(T));
    const int grid = std::min(c->nsub, c->jac_grid);
#define GDSW_JAC_LAUNCH(TS, MODE)                                                                         \
  k_local_jac<T, TS, MODE><<<grid, c->jac_threads, shm, s>>>(                                            \
      r, c->om_ptr, c->om_dofs, c->jac_stream, c->jac_off16, c->jac_bytes,                               \
      static_cast<int>(jac_slot_a(c, c->jac_mode)), static_cast<int>(jac_slot_b(c, c->jac_mode)),        \
      c->max_m, c->nsub, c->opt.sweeps_trsv, zl, ks, c->derr, c->wait_cycles, gate, c->stall_test)
    if (c->fp16) {
      if constexpr (std::is_same<T, float>::value) {
        if (c->jac_mode == 2) GDSW_JAC_LAUNCH(__half, 2); else GDSW_JAC_LAUNCH(__half, 1);
      }
    } else {
      if (c->jac_mode == 2) GDSW_JAC_LAUNCH(T, 2); else GDSW_JAC_LAUNCH(T, 1);
    }
#undef GDSW_JAC_LAUNCH
  } else {
    const int jac = c->opt.trsv == GDSW_TRSV_JACOBI;
    const size_t shm = size_t(c->max_m) * sizeof(T) * (jac ? 3 : 1);
    k_local_tri<T><<<c->nsub, c->tri_threads, shm, s>>>(r, c->om_ptr, c->om_dofs, ell<T>(c, true),
                                             ell<T>(c, false), jac, c->opt.sweeps_trsv, zl, ks, gate);
  }
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

template <class T>
gdsw_status launch_phiT(Ctx* c, const double* r, cudaStream_t s, const KrylovScalars* ks, const BatchGate& gate) {
  if (c->n0 == 0) return GDSW_OK;
  if (c->n_chunks == 0) return GDSW_OK;
  const int grid = c->n_cta_chunks + (c->n_chunks - c->n_cta_chunks + 7) / 8;
  if (c->phiT_wide)
    k_phiT<T, true><<<grid, 256, 0, s>>>(c->n_chunks, c->n_cta_chunks, r, c->brow_ptr, c->brow_dof, c->bcol_ptr,
                                         c->phi_off, static_cast<const T*>(c->phi), c->chunk_blk, c->chunk_r0,
                                         c->chunk_r1, c->chunk_slot, c->partial, ks, gate);
  else
    k_phiT<T, false><<<grid, 256, 0, s>>>(c->n_chunks, c->n_cta_chunks, r, c->brow_ptr, c->brow_dof, c->bcol_ptr,
                                          c->phi_off, static_cast<const T*>(c->phi), c->chunk_blk, c->chunk_r0,
                                          c->chunk_r1, c->chunk_slot, c->partial, ks, gate);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

// Phi y beside the local solves reads y through the block-column map where
// the blocks are narrow (no slot gather launched); a fixed rule, as the form
// of Phi^T r it follows.
inline bool prolong_via_map(const Ctx* c) { return c->prolong && !c->phiT_wide; }

gdsw_status launch_coarse(Ctx* c, cudaStream_t s, const KrylovScalars* ks, const BatchGate& gate) {
  if (c->n0 == 0) return GDSW_OK;
  k_coarse_c<<<(c->n0 + 255) / 256, 256, 0, s>>>(c->n0, c->cs_ptr, c->cs_idx, c->partial, c->cvec, c->cvec32,
                                                  ks, gate);
  const int grid = std::min((c->n0 + 3) / 4, kNumSMs * 8);
  if (c->A0inv32 != nullptr)
    k_coarse_gemv<float><<<grid, 256, 0, s>>>(c->n0, c->A0inv32, c->coarse_prob, c->prob_c0, c->a0_off,
                                              c->cvec32, c->yvec, c->yvec32, ks, gate);
  else
    k_coarse_gemv<double><<<grid, 256, 0, s>>>(c->n0, c->A0inv, c->coarse_prob, c->prob_c0, c->a0_off,
                                               c->cvec, c->yvec, c->yvec32, ks, gate);
  // y at every block-column slot, for the scatter-add's Phi y or for
  // k_prolong on wide blocks
  if (c->n_bslots > 0 && !prolong_via_map(c)) {
    const int sg = std::min((c->n_bslots + 255) / 256, kNumSMs * 4);
    if (c->fp32)
      k_coarse_slots<float><<<sg, 256, 0, s>>>(c->n_bslots, c->bcol, c->yvec32, static_cast<float*>(c->yslot), ks);
    else
      k_coarse_slots<double><<<sg, 256, 0, s>>>(c->n_bslots, c->bcol, c->yvec, static_cast<double*>(c->yslot), ks);
  }
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

template <class T>
gdsw_status launch_prolong(Ctx* c, cudaStream_t s, const KrylovScalars* ks, const BatchGate& gate) {
  if (!c->prolong) return GDSW_OK;
  const int grid = std::max(1, std::min((c->n + 255) / 256, kNumSMs * 8));
  k_prolong<T><<<grid, 256, 0, s>>>(c->n, c->pos_blk, c->brow_ptr, c->bcol_ptr, c->phi_off,
                                    static_cast<const T*>(c->phi), prolong_via_map(c) ? c->bcol : nullptr,
                                    !prolong_via_map(c) ? static_cast<const T*>(c->yslot)
                                    : c->fp32 ? reinterpret_cast<const T*>(c->yvec32)
                                              : reinterpret_cast<const T*>(c->yvec),
                                    static_cast<T*>(c->ubuf), ks, gate);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

template <class T>
gdsw_status launch_combine(Ctx* c, const double* r, double* z, cudaStream_t s, bool dots, bool gated,
                           const BatchGate& gate) {
  const int grid = std::max(1, std::min(c->combine_cb == 8 && !c->prolong ? c->combine_grid8 : c->combine_grid,
                                        (c->n + 255) / 256));
#define GDSW_COMBINE_LAUNCH(CBB, PP)                                                                        \
  k_combine<T, 2, CBB, PP><<<grid, 256, 0, s>>>(c->n, r, z, c->brow_dof, c->pos_blk, c->brow_ptr, c->bcol_ptr,  \
                                                c->phi_off, static_cast<const T*>(c->phi),                     \
                                                static_cast<const T*>(c->yslot), static_cast<const T*>(c->ubuf), \
                                                c->pull_ptr, c->pull_pos, static_cast<const T*>(c->zloc),      \
                                                dots ? (c->flexible ? 2 : 1) : 0, c->red,                      \
                                                (dots || gated) ? c->ks : nullptr, gate)
  if (c->prolong) GDSW_COMBINE_LAUNCH(4, true);
  else if (c->combine_cb == 8) GDSW_COMBINE_LAUNCH(8, false);
  else GDSW_COMBINE_LAUNCH(4, false);
#undef GDSW_COMBINE_LAUNCH
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

// dots: the PCG form (z, (r, z) and beta into the Krylov scalars); gated:
// every kernel returns at once when the Krylov loop has set its stop flag.
template <class T>
gdsw_status apply_t(Ctx* c, const double* r, double* z, cudaStream_t s, bool dots, bool gated, cudaEvent_t* ev,
                    bool batch = false) {
  const KrylovScalars* ks = (dots || gated) ? c->ks : nullptr;
  const BatchGate gate = batch ? batch_gate(c) : BatchGate{};
  if (ev == nullptr && c->n0 > 0 && c->aux_stream != nullptr) {
    // The one-level and coarse branches of Eq. 1 are independent until the
    // final sum: the coarse branch (Phi^T r, c, A0^-1 c) runs on a second
    // stream beside the local solves and joins before the scatter-add.
    GDSW_CK(cudaEventRecord(c->ev_fork, s));
    GDSW_CK(cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0));
    GDSW_TRY(launch_phiT<T>(c, r, c->aux_stream, ks, gate));
    GDSW_TRY(launch_coarse(c, c->aux_stream, ks, gate));
    GDSW_TRY(launch_prolong<T>(c, c->aux_stream, ks, gate));
    GDSW_CK(cudaEventRecord(c->ev_join, c->aux_stream));
    GDSW_TRY(launch_local<T>(c, r, s, ks, gate));
    GDSW_CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    GDSW_TRY(launch_combine<T>(c, r, z, s, dots, gated, gate));
    return GDSW_OK;
  }
  if (ev) GDSW_CK(cudaEventRecord(ev[0], s));
  GDSW_TRY(launch_local<T>(c, r, s, ks, gate));
  if (ev) GDSW_CK(cudaEventRecord(ev[1], s));
  GDSW_TRY(launch_phiT<T>(c, r, s, ks, gate));
  if (ev) GDSW_CK(cudaEventRecord(ev[2], s));
  GDSW_TRY(launch_coarse(c, s, ks, gate));
  GDSW_TRY(launch_prolong<T>(c, s, ks, gate));
  if (ev) GDSW_CK(cudaEventRecord(ev[3], s));
  GDSW_TRY(launch_combine<T>(c, r, z, s, dots, gated, gate));
  if (ev) GDSW_CK(cudaEventRecord(ev[4], s));
  return GDSW_OK;
}

}  // namespace

// Resident CTAs per SM of the pipelined local solve for this handle's types,
// ring depth S and dynamic shared memory (0 when it does not fit).  Raises the
// kernel's dynamic shared memory limit first.
template <class TT, class TS, int TP>
gdsw_status pipe_occupancy_t(int S, bool sf, size_t shm, int threads, int* per_sm) {
  *per_sm = 0;
  auto one = [&](auto kernel) -> gdsw_status {
    GDSW_CK(allow_max_dynamic_smem(kernel));
    cudaFuncAttributes fa;
    GDSW_CK(cudaFuncGetAttributes(&fa, kernel));
    if (shm + fa.sharedSizeBytes > size_t(max_block_smem_optin())) return GDSW_OK;
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, shm));
    return GDSW_OK;
  };
  if (sf) {
    switch (S) {
      case 2: return one(k_local_sf<TT, TS, 2>);
      case 4: return one(k_local_sf<TT, TS, 4>);
      case 8: return one(k_local_sf<TT, TS, 8>);
      default: return one(k_local_sf<TT, TS, 16>);
    }
  }
  switch (S) {
    case 2: return one(k_local_pipe<TT, TS, 2, TP>);
    case 4: return one(k_local_pipe<TT, TS, 4, TP>);
    case 8: return one(k_local_pipe<TT, TS, 8, TP>);
    default: return one(k_local_pipe<TT, TS, 16, TP>);
  }
}

// Dynamic shared memory of the pipelined local solve with ring depth S.
size_t pipe_smem(const Ctx* c, int S, bool sf) {
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  return size_t(S) * c->rec_stage_bytes + pipe_vector_bytes(c->max_m, es) + (sf ? sf_flag_bytes(c->max_m) : 0);
}

gdsw_status pipe_occupancy(const Ctx* c, int S, bool sf, int* per_sm) {
  const size_t shm = pipe_smem(c, S, sf);
  const int th = c->rec_consumers + 32;
  if (c->fp16)
    return c->rec_tpr == 8 ? pipe_occupancy_t<float, __half, 8>(S, sf, shm, th, per_sm)
                           : pipe_occupancy_t<float, __half, 1>(S, sf, shm, th, per_sm);
  if (c->fp32)
    return c->rec_tpr == 8 ? pipe_occupancy_t<float, float, 8>(S, sf, shm, th, per_sm)
                           : pipe_occupancy_t<float, float, 1>(S, sf, shm, th, per_sm);
  return c->rec_tpr == 8 ? pipe_occupancy_t<double, double, 8>(S, sf, shm, th, per_sm)
                         : pipe_occupancy_t<double, double, 1>(S, sf, shm, th, per_sm);
}

// Resident CTAs per SM of the row-program solve with D slots per thread
// (raises its dynamic shared memory limit first; 0 when it does not fit).
gdsw_status steps_occupancy(Ctx* c, int D, int* per_sm) {
  const size_t shm = steps_smem_bytes(D, c->step_max, c->max_m);
  *per_sm = 0;
  if (shm > size_t(max_block_smem_optin())) return GDSW_OK;
  switch (D) {
    case 4:
      GDSW_CK(allow_max_dynamic_smem(k_local_steps<4>));
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_local_steps<4>, kStepRows, shm));
      break;
    case 12:
      GDSW_CK(allow_max_dynamic_smem(k_local_steps<12>));
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_local_steps<12>, kStepRows, shm));
      break;
    default:
      GDSW_CK(allow_max_dynamic_smem(k_local_steps<8>));
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_local_steps<8>, kStepRows, shm));
      break;
  }
  return GDSW_OK;
}

// Resident CTAs per SM of the node-program solve with S ring slots, NT
// threads and LPN lanes per node (raises
// its dynamic shared memory limit first; 0 when it does not fit).
gdsw_status nodes_occupancy(Ctx* c, int S, int NT, int LPN, int* per_sm) {
  const size_t shm = nodes_smem_bytes(S, c->node_slot_bytes, c->max_m);
  *per_sm = 0;
  if (S < 2 || S > kNodeSlots || shm > size_t(max_block_smem_optin())) return GDSW_OK;
#define GDSW_NODES_OCC(TT, LL)                                                                \
  do {                                                                                        \
    GDSW_CK(allow_max_dynamic_smem(k_local_nodes<TT, LL>));                                   \
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_local_nodes<TT, LL>, TT, shm)); \
  } while (0)
  const int sel = (NT == 256 ? 0 : 3) + (LPN == 2 ? 0 : LPN == 4 ? 1 : 2);
  switch (sel) {
    case 0: GDSW_NODES_OCC(256, 2); break;
    case 1: GDSW_NODES_OCC(256, 4); break;
    case 2: GDSW_NODES_OCC(256, 8); break;
    case 3: GDSW_NODES_OCC(512, 2); break;
    case 4: GDSW_NODES_OCC(512, 4); break;
    default: GDSW_NODES_OCC(512, 8); break;
  }
#undef GDSW_NODES_OCC
  return GDSW_OK;
}

// The scatter-add with 4 and with 8 Phi columns per trip, three launches each
// (CUDA events, after one warm-up, without the dots) on scratch vectors; the
// faster is kept.  Both form every sum in the same order.
gdsw_status tune_combine(Ctx* c) {
  cudaStream_t s;
  GDSW_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  double* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gdsw_status st = GDSW_OK;
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * 2 * size_t(c->n));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(double) * 2 * size_t(c->n), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float t[2] = {0.f, 0.f};
  for (int k = 0; k < 2 && e == cudaSuccess && st == GDSW_OK; ++k) {
    c->combine_cb = k == 0 ? 4 : 8;
    st = c->fp32 ? launch_combine<float>(c, buf, buf + c->n, s, false, false, BatchGate{})
                 : launch_combine<double>(c, buf, buf + c->n, s, false, false, BatchGate{});
    e = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep)
      st = c->fp32 ? launch_combine<float>(c, buf, buf + c->n, s, false, false, BatchGate{})
                   : launch_combine<double>(c, buf, buf + c->n, s, false, false, BatchGate{});
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], e0, e1);
  }
  if (e != cudaSuccess && st == GDSW_OK) {
    set_error("scatter-add tuning: %s", cudaGetErrorString(e));
    st = GDSW_ERR_CUDA;
  }
  c->combine_cb = t[1] < t[0] ? 8 : 4;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  cudaStreamDestroy(s);
  return st;
}

// Measured choice of the pipelined local solve's shape: every ring depth that
// fits, with 128 to 992 consumer threads, timed over three launches each
// (CUDA events, after one warm-up launch) on a zero right-hand side, and the
// unpipelined level-scheduled kernel beside them; the fastest is kept.  Every
// candidate computes the same values in the same order, so the choice changes
// the speed only, never the result.
gdsw_status tune_local(Ctx* c) {
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  // timed with the default wait bound, whatever the handle's
  const long long keep_wait = c->wait_cycles;
  c->wait_cycles = kDefaultWaitCycles;
  cudaStream_t s;
  GDSW_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  double* r = nullptr;
  cudaEvent_t e0, e1;
  gdsw_status st = GDSW_OK;
  auto fail = [&](cudaError_t e) { set_error("local-solve tuning: %s", cudaGetErrorString(e)); st = GDSW_ERR_CUDA; };
  cudaError_t e = cudaMalloc(&r, sizeof(double) * std::max(1, c->n));
  if (e == cudaSuccess) e = cudaMemsetAsync(r, 0, sizeof(double) * std::max(1, c->n), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) fail(e);
  const int keep_s = c->rec_stages, keep_nt = c->rec_consumers;
  float best = 3.4e38f;
  int best_s = keep_s, best_nt = keep_nt;
  bool best_sf = false;
  const int cand[4] = {16, 8, 4, 2};
  // the barrier-free kernel takes rows of up to 8 entries (one thread per row)
  const int n_kinds = c->rec_tpr == 1 ? 2 : 1;
  for (int kind = 0; kind < n_kinds && st == GDSW_OK; ++kind)
  for (int q = 0; q < 4 && st == GDSW_OK; ++q) {
    for (int nt : {64, 128, 256, 512}) {
      if (c->rec_tpr == 8 && nt < 256) continue;
      c->rec_stages = cand[q];
      c->rec_consumers = nt;
      c->rec_sf = kind == 1;
      int per_sm = 0;
      st = pipe_occupancy(c, cand[q], c->rec_sf, &per_sm);
      if (st != GDSW_OK) break;
      if (per_sm == 0) continue;
      st = c->fp32 ? launch_local<float>(c, r, s, nullptr, BatchGate{}) : launch_local<double>(c, r, s, nullptr, BatchGate{});
      if (st != GDSW_OK) break;
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep)
        st = c->fp32 ? launch_local<float>(c, r, s, nullptr, BatchGate{}) : launch_local<double>(c, r, s, nullptr, BatchGate{});
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) { fail(e); break; }
      if (ms < best) { best = ms; best_s = cand[q]; best_nt = nt; best_sf = c->rec_sf; }
    }
  }
  c->rec_sf = false;
  // the row-program kernel with 4, 8 or 12 steps in flight per thread
  int best_depth = 0;
  if (c->steps != nullptr && c->fp32 && !c->fp16) {
    for (int D : {4, 8, 12}) {
      if (st != GDSW_OK) break;
      int per_sm = 0;
      st = steps_occupancy(c, D, &per_sm);
      if (st != GDSW_OK || per_sm == 0) continue;
      c->step_depth = D;
      st = launch_local<float>(c, r, s, nullptr, BatchGate{});
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep) st = launch_local<float>(c, r, s, nullptr, BatchGate{});
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) { fail(e); break; }
      if (ms < best) { best = ms; best_depth = D; }
    }
    c->step_depth = 0;
  }
  // the node-program kernel with 2 to 4 ring slots
  int best_nodes = 0, best_node_nt = kNodeThreads, best_node_lanes = 4;
  if (c->node_stream != nullptr && c->fp32 && !c->fp16) {
    for (int S : {2, 4, 6})
    for (int NT : {256, 512})
    for (int LPN : {2, 4, 8}) {
      if (st != GDSW_OK) break;
      int per_sm = 0;
      st = nodes_occupancy(c, S, NT, LPN, &per_sm);
      if (st != GDSW_OK || per_sm == 0) continue;
      c->node_stages = S;
      c->node_threads = NT;
      c->node_lanes = LPN;
      st = launch_local<float>(c, r, s, nullptr, BatchGate{});
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep) st = launch_local<float>(c, r, s, nullptr, BatchGate{});
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) { fail(e); break; }
      if (ms < best) { best = ms; best_nodes = S; best_node_nt = NT; best_node_lanes = LPN; best_depth = 0; }
    }
    c->node_stages = 0;
  }
  // the unpipelined level-scheduled kernel (factors read through L2), with
  // 256 to 1024 threads, as further candidates
  int best_tri = c->tri_threads;
  for (int tt : {256, 512, 1024}) {
    if (st != GDSW_OK) break;
    c->rec_stages = 0;
    c->tri_threads = tt;
    st = c->fp32 ? launch_local<float>(c, r, s, nullptr, BatchGate{}) : launch_local<double>(c, r, s, nullptr, BatchGate{});
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep)
      st = c->fp32 ? launch_local<float>(c, r, s, nullptr, BatchGate{}) : launch_local<double>(c, r, s, nullptr, BatchGate{});
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { fail(e); break; }
    if (ms < best) { best = ms; best_s = 0; best_tri = tt; best_depth = 0; best_nodes = 0; }
  }
  c->step_depth = best_depth;
  c->node_stages = best_nodes;
  c->node_threads = best_node_nt;
  c->node_lanes = best_node_lanes;
  c->rec_stages = best_s;
  c->rec_consumers = best_nt;
  c->rec_sf = best_s > 0 && best_sf;
  c->tri_threads = best_s == 0 ? best_tri : 256;
  c->wait_cycles = keep_wait;
  if (r) cudaFree(r);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st == GDSW_OK) st = check_device_errors(c, nullptr);
  return st;
}

// Resident CTAs per SM of the resident-block Jacobi kernel (raises its
// dynamic shared memory limit first; 0 when it does not fit).
template <class TT, class TS>
gdsw_status jac_occupancy_t(int mode, size_t shm, int threads, int* per_sm) {
  *per_sm = 0;
  auto one = [&](auto kernel) -> gdsw_status {
    GDSW_CK(allow_max_dynamic_smem(kernel));
    cudaFuncAttributes fa;
    GDSW_CK(cudaFuncGetAttributes(&fa, kernel));
    if (shm + fa.sharedSizeBytes > size_t(max_block_smem_optin())) return GDSW_OK;
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, shm));
    return GDSW_OK;
  };
  return mode == 2 ? one(k_local_jac<TT, TS, 2>) : one(k_local_jac<TT, TS, 1>);
}

gdsw_status jac_occupancy(const Ctx* c, int mode, size_t shm, int threads, int* per_sm) {
  if (c->fp16) return jac_occupancy_t<float, __half>(mode, shm, threads, per_sm);
  if (c->fp32) return jac_occupancy_t<float, float>(mode, shm, threads, per_sm);
  return jac_occupancy_t<double, double>(mode, shm, threads, per_sm);
}

// Threads of the resident-block Jacobi solve, chosen by timing (three launches
// each after a warm-up, on a zero right-hand side); every choice computes the
// same values.
gdsw_status tune_jacobi(Ctx* c) {
  cudaStream_t s;
  GDSW_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  double* r = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gdsw_status st = GDSW_OK;
  cudaError_t e = cudaMalloc(&r, sizeof(double) * std::max(1, c->n));
  if (e == cudaSuccess) e = cudaMemsetAsync(r, 0, sizeof(double) * std::max(1, c->n), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { set_error("Jacobi tuning: %s", cudaGetErrorString(e)); st = GDSW_ERR_CUDA; }
  float best = 3.4e38f;
  int best_t = c->jac_threads;
  for (int th : {256, 512, 1024}) {
    if (st != GDSW_OK) break;
    c->jac_threads = th;
    auto one = [&]() {
      return c->fp32 ? launch_local<float>(c, r, s, nullptr, BatchGate{})
                     : launch_local<double>(c, r, s, nullptr, BatchGate{});
    };
    st = one();
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && st == GDSW_OK; ++rep) st = one();
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { set_error("Jacobi tuning: %s", cudaGetErrorString(e)); st = GDSW_ERR_CUDA; break; }
    if (ms < best) { best = ms; best_t = th; }
  }
  c->jac_threads = best_t;
  if (r) cudaFree(r);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st == GDSW_OK) st = check_device_errors(c, nullptr);
  return st;
}

gdsw_status apply_configure(Ctx* c) {
  const char* two = getenv("GDSW_APPLY_STREAMS");
  if (c->aux_stream == nullptr && (two == nullptr || two[0] != '1')) {
    GDSW_CK(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
    GDSW_CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    GDSW_CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    GDSW_CK(cudaEventCreateWithFlags(&c->ev_x, cudaEventDisableTiming));
    GDSW_CK(cudaEventCreateWithFlags(&c->ev_xdone, cudaEventDisableTiming));
  }
  if (c->derr == nullptr) {
    GDSW_TRY(dalloc(c, &c->derr, 4));
    GDSW_CK(cudaMemset(c->derr, 0, 4 * sizeof(int)));
  }
  // kernels that may need more than 48 KB of dynamic shared memory
  const int jac = c->opt.trsv == GDSW_TRSV_JACOBI;
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  const size_t shm_local = size_t(c->max_m) * es * (c->opt.local_solver == GDSW_LOCAL_EXACT ? 1 : (jac ? 3 : 1));
  if (shm_local > 227 * 1024) {
    set_error("subdomain of %d unknowns does not fit the local solve's shared memory", c->max_m);
    return GDSW_ERR_UNSUPPORTED;
  }
  // pipelined level-scheduled solve: the ring depth (16, 8, 4 or 2 stages)
  // that runs all subdomains in the fewest waves of resident CTAs (one CTA per
  // subdomain; the local solve is latency-bound, so a wave that is only partly
  // filled costs as much as a full one), the deepest ring among those
  c->rec_stages = 0;
  c->rec_tpr = c->rec_max_width > 8 ? 8 : 1;
  // consumer threads: 128 when a level has at most 256 rows to update (two per
  // thread at most), which halves the instructions that idle threads spend per
  // level; 256 for wider levels or threads-per-row groups
  c->rec_consumers = (c->rec_tpr == 1 && c->rec_max_rows <= 256) ? 128 : 256;
  const char* env = getenv("GDSW_LOCAL_PIPE");
  const bool pipe_ok = (env == nullptr || env[0] != '0') && c->rec_stream != nullptr &&
                       c->opt.local_solver != GDSW_LOCAL_EXACT && !jac;
  if (pipe_ok) {
    int dev = 0, sms = 148;
    GDSW_CK(cudaGetDevice(&dev));
    GDSW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int depth_env = getenv("GDSW_PIPE_STAGES") ? atoi(getenv("GDSW_PIPE_STAGES")) : 0;
    const int cand[4] = {16, 8, 4, 2};
    int64_t best_waves = INT64_MAX;
    for (int q = 0; q < 4; ++q) {
      if (depth_env > 0 && cand[q] != depth_env) continue;
      int per_sm = 0;
      GDSW_TRY(pipe_occupancy(c, cand[q], false, &per_sm));
      if (per_sm == 0) continue;
      const int64_t waves = (int64_t(c->nsub) + int64_t(sms) * per_sm - 1) / (int64_t(sms) * per_sm);
      if (waves < best_waves) {
        best_waves = waves;
        c->rec_stages = cand[q];
      }
    }
  }
  if (c->fp32) {
    GDSW_CK(allow_max_dynamic_smem(k_local_tri<float>));
    GDSW_CK(allow_max_dynamic_smem(k_local_dense<float>));
  } else {
    GDSW_CK(allow_max_dynamic_smem(k_local_tri<double>));
    GDSW_CK(allow_max_dynamic_smem(k_local_dense<double>));
  }
  // resident-block Jacobi sweeps: mode 2 when an L and a U block fit beside
  // the vectors, else mode 1; GDSW_JACOBI_RESIDENT=0 keeps the unpipelined
  // Jacobi kernel (which reads the factors from L2/HBM on every sweep)
  c->jac_mode = 0;
  if (c->jac_stream != nullptr && !(getenv("GDSW_JACOBI_RESIDENT") && getenv("GDSW_JACOBI_RESIDENT")[0] == '0')) {
    int dev = 0, sms = kNumSMs;
    GDSW_CK(cudaGetDevice(&dev));
    GDSW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int force = getenv("GDSW_JACOBI_MODE") ? atoi(getenv("GDSW_JACOBI_MODE")) : 0;
    for (int mode : {2, 1}) {
      if (force != 0 && mode != force) continue;
      const size_t shm = jac_smem(c, mode, es);
      int per_sm = 0;
      GDSW_TRY(jac_occupancy(c, mode, shm, c->jac_threads, &per_sm));
      if (per_sm > 0) {
        c->jac_mode = mode;
        c->jac_grid = sms * per_sm;
        break;
      }
    }
    if (c->jac_mode > 0 && c->opt.autotune && !getenv("GDSW_LOCAL_SHAPE")) GDSW_TRY(tune_jacobi(c));
    if (const char* e = getenv("GDSW_LOCAL_SHAPE")) {
      int st = 0, nt = 0;
      if (sscanf(e, "%d,%d", &st, &nt) == 2 && (nt == 256 || nt == 512 || nt == 1024)) c->jac_threads = nt;
    }
  }
  // records prefetched into L2 ahead of the ring (bytes per subdomain);
  // GDSW_PIPE_PREFETCH overrides the default
  c->rec_prefetch = 0;
  if (const char* e = getenv("GDSW_PIPE_PREFETCH")) c->rec_prefetch = std::max(0, atoi(e)) & ~15;
  // GDSW_TEST_STALL=1: the failure test of the bounded waits (see k_local_pipe)
  if (const char* e = getenv("GDSW_TEST_STALL")) c->stall_test = e[0] == '1';
  // GDSW_LOCAL_SHAPE="stages,threads[,kind]" fixes the shape instead of
  // timing it (for profilers, under which the timings mean nothing, and for
  // the failure tests); kind 1 selects the solve without a barrier per level,
  // kind 2 the row programs with `stages` steps in flight per thread, kind 3
  // the node programs with `stages` ring slots, 256 or 512 threads and a
  // fourth field of 2, 4 (default) or 8 lanes per node
  const char* shape = getenv("GDSW_LOCAL_SHAPE");
  if (c->rec_stages > 0 && shape != nullptr) {
    int st = 0, nt = 0, sf = 0, lanes = 4;
    const int got = sscanf(shape, "%d,%d,%d,%d", &st, &nt, &sf, &lanes);
    if (got >= 3 && sf == 3 && c->node_stream != nullptr && st >= 2 && st <= kNodeSlots &&
        (nt == 256 || nt == 512) && (lanes == 2 || lanes == 4 || lanes == 8)) {
      int per_sm = 0;
      GDSW_TRY(nodes_occupancy(c, st, nt, lanes, &per_sm));
      if (per_sm == 0) {
        set_error("GDSW_LOCAL_SHAPE=%s does not fit the shared memory", shape);
        return GDSW_ERR_UNSUPPORTED;
      }
      c->node_stages = st;
      c->node_threads = nt;
      c->node_lanes = lanes;
    } else if (got == 3 && sf == 2 && c->steps != nullptr && c->fp32 && !c->fp16 && (st == 4 || st == 8 || st == 12)) {
      int per_sm = 0;
      GDSW_TRY(steps_occupancy(c, st, &per_sm));
      if (per_sm == 0) {
        set_error("GDSW_LOCAL_SHAPE=%s does not fit the shared memory", shape);
        return GDSW_ERR_UNSUPPORTED;
      }
      c->step_depth = st;
    } else if (got >= 2 && got <= 3 && (st == 0 || st == 2 || st == 4 || st == 8 || st == 16) &&
        (nt == 64 || nt == 128 || nt == 256 || nt == 512 || nt == 1024)) {
      c->rec_stages = st;
      if (st > 0) c->rec_consumers = nt == 1024 ? 512 : nt; else c->tri_threads = nt;
      c->rec_sf = st > 0 && got == 3 && sf == 1 && c->rec_tpr == 1;
      int per_sm = 0;
      if (st > 0) GDSW_TRY(pipe_occupancy(c, st, c->rec_sf, &per_sm));
      if (st > 0 && per_sm == 0) {
        set_error("GDSW_LOCAL_SHAPE=%s does not fit the shared memory", shape);
        return GDSW_ERR_UNSUPPORTED;
      }
    }
  } else if (c->rec_stages > 0 && c->opt.autotune && !c->stall_test) {
    GDSW_TRY(tune_local(c));
  }
  // the scatter-add is a grid-stride loop: exactly the CTAs that are resident at once
  {
    int dev = 0, sms = kNumSMs, per_sm = 1;
    GDSW_CK(cudaGetDevice(&dev));
    GDSW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm8 = 1;
    if (c->fp32) {
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_combine<float, 2, 4, false>, 256, 0));
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm8, k_combine<float, 2, 8, false>, 256, 0));
    } else {
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_combine<double, 2, 4, false>, 256, 0));
      GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm8, k_combine<double, 2, 8, false>, 256, 0));
    }
    c->combine_grid = std::max(1, per_sm) * sms;
    c->combine_grid8 = std::max(1, per_sm8) * sms;
  }
  // Phi y beside the local solves (k_prolong on the coarse stream, one value
  // per block-row position), the scatter-add then only adding it: for one
  // problem (not a batch, whose members stop at different iterations) when
  // the local solves leave SMs idle (fewer subdomains than SMs, one CTA each)
  // and the problem is large enough that one more launch per apply does not
  // matter (n >= 65,536), or when the problem is so large (n >= 2^20) that
  // the local solves outlast the coarse branch with the product added to it
  // (a fixed rule, so a handle's rounding never depends on a timing).
  // GDSW_PROLONG=1 or 0 forces it on or off.
  c->prolong = 0;
  bool want_prolong = false;
  {
    int dev = 0, sms = kNumSMs;
    GDSW_CK(cudaGetDevice(&dev));
    GDSW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    want_prolong = c->nprob == 1 && (c->nsub < sms ? c->n >= 65536 : c->n >= (1 << 20));
    if (const char* e = getenv("GDSW_PROLONG")) want_prolong = e[0] == '1';
  }
  if (c->n0 > 0 && want_prolong) {
    if (c->fp32) GDSW_TRY(dalloc(c, reinterpret_cast<float**>(&c->ubuf), c->n));
    else GDSW_TRY(dalloc(c, reinterpret_cast<double**>(&c->ubuf), c->n));
    c->prolong = 1;
  }
  // Phi columns per trip of the scatter-add: 4 (more CTAs per SM, for many
  // positions per thread) or 8 (more loads in flight, for wide Phi blocks),
  // timed; GDSW_COMBINE_CB=4 or 8 fixes it
  c->combine_cb = 4;
  if (const char* e = getenv("GDSW_COMBINE_CB")) {
    c->combine_cb = atoi(e) == 8 ? 8 : 4;
  } else if (c->opt.autotune && !c->stall_test && c->n > 0 && !c->mf && !c->prolong) {
    GDSW_TRY(tune_combine(c));
  }
  return GDSW_OK;
}

// Reads (and clears) the device error flags; a bounded wait that ran out is
// reported as GDSW_ERR_TIMEOUT.
gdsw_status check_device_errors(Ctx* c, cudaStream_t s) {
  int h = 0;
  GDSW_CK(cudaMemcpyAsync(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  GDSW_CK(cudaStreamSynchronize(s));
  if (h != 0) {
    GDSW_CK(cudaMemsetAsync(c->derr, 0, sizeof(int), s));
    set_error("a bounded device wait in the local solve ran out");
    return GDSW_ERR_TIMEOUT;
  }
  return GDSW_OK;
}

gdsw_status apply_enqueue(Ctx* c, const double* r, double* z, cudaStream_t s, bool rz_dots) {
  return c->fp32 ? apply_t<float>(c, r, z, s, rz_dots, false, nullptr)
                 : apply_t<double>(c, r, z, s, rz_dots, false, nullptr);
}

BatchGate batch_gate(const Ctx* c) {
  BatchGate g{};
  if (c->nprob > 1 && c->bks != nullptr && c->sub_prob != nullptr) {
    g.bs = c->bks;
    g.sub_prob = c->sub_prob;
    g.blk_prob = c->blk_prob;
    g.col_prob = c->coarse_prob;
    g.row_ptr = c->prob_rows;
    g.nprob = c->nprob;
  }
  return g;
}

gdsw_status apply_enqueue_batch(Ctx* c, const double* r, double* z, cudaStream_t s) {
  return c->fp32 ? apply_t<float>(c, r, z, s, false, false, nullptr, true)
                 : apply_t<double>(c, r, z, s, false, false, nullptr, true);
}

gdsw_status apply_enqueue_gated(Ctx* c, const double* r, double* z, cudaStream_t s) {
  return c->fp32 ? apply_t<float>(c, r, z, s, false, true, nullptr)
                 : apply_t<double>(c, r, z, s, false, true, nullptr);
}

gdsw_status apply_timed_dots(Ctx* c, const double* r, double* z, cudaStream_t s, cudaEvent_t* ev) {
  return c->fp32 ? apply_t<float>(c, r, z, s, true, false, ev) : apply_t<double>(c, r, z, s, true, false, ev);
}

gdsw_status apply_timed(Ctx* c, const double* r, double* z, cudaStream_t s, double* ms) {
  GDSW_TRY(c->fp32 ? apply_t<float>(c, r, z, s, false, false, c->ev)
                   : apply_t<double>(c, r, z, s, false, false, c->ev));
  GDSW_CK(cudaEventSynchronize(c->ev[4]));
  GDSW_TRY(check_device_errors(c, s));
  for (int q = 0; q < 4; ++q) {
    float t = 0.f;
    GDSW_CK(cudaEventElapsedTime(&t, c->ev[q], c->ev[q + 1]));
    ms[q] = t;
  }
  return GDSW_OK;
}

// The persistent PCG kernel for this handle, or none: PCG on one problem with
// dense exact local solves and at most kPersistMaxN0 coarse columns, when
// GDSW_PERSISTENT=1 asks for it (measured slower than the graph-launched loop
// on the Poisson 16^3 workload, 1.44 against 1.11 ms per solve: every phase
// runs on one CTA per SM and waits at a grid barrier, where the graph's kernels
// each fill the GPU).  Sets the unit table, the barrier counter and the
// cooperative grid (every CTA resident at once, kPersistPerSM per SM).
gdsw_status persistent_configure(Ctx* c) {
  c->persist_grid = 0;
  const char* e = getenv("GDSW_PERSISTENT");
  if (e == nullptr || e[0] != '1') return GDSW_OK;
  if (c->opt.krylov != GDSW_KRYLOV_PCG || c->nprob != 1 || c->mf || c->ainv == nullptr ||
      c->opt.local_solver != GDSW_LOCAL_EXACT || c->n0 < 1 || c->n0 > kPersistMaxN0 || c->n <= 0)
    return GDSW_OK;
  std::vector<int> om(size_t(c->nsub) + 1);
  GDSW_CK(cudaMemcpy(om.data(), c->om_ptr, sizeof(int) * om.size(), cudaMemcpyDeviceToHost));
  std::vector<int> up(size_t(c->nsub) + 1, 0);
  for (int q = 0; q < c->nsub; ++q) up[q + 1] = up[q] + (om[q + 1] - om[q] + kDenseRows - 1) / kDenseRows;
  GDSW_TRY(upload(c, &c->unit_ptr, up, nullptr));
  c->n_units = up[c->nsub];
  if (c->pbar == nullptr) GDSW_TRY(dalloc(c, &c->pbar, 1));
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  c->persist_smem = ((size_t(c->max_m) * es + 15) & ~size_t(15)) + 2 * kPersistMaxN0 * es;
  int dev = 0, sms = kNumSMs, per_sm = 0;
  GDSW_CK(cudaGetDevice(&dev));
  GDSW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (c->fp32) {
    GDSW_CK(allow_max_dynamic_smem(k_pcg_persistent<float>));
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<float>, 256, c->persist_smem));
  } else {
    GDSW_CK(allow_max_dynamic_smem(k_pcg_persistent<double>));
    GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<double>, 256, c->persist_smem));
  }
  if (per_sm <= 0) return GDSW_OK;
  // the reduction buffer holds four partials per CTA
  c->persist_grid = std::min(std::min(per_sm, kPersistPerSM) * sms, (c->red_len - 64) / 4);
  return GDSW_OK;
}

// PCG iterations from the current state until the stopping test holds, as one
// cooperative launch (see k_pcg_persistent); the state stays in the handle's
// Krylov workspace and scalars exactly as after the graph loop.
gdsw_status pcg_persistent_run(Ctx* c, cudaStream_t s) {
  GDSW_CK(cudaMemsetAsync(c->pbar, 0, sizeof(unsigned), s));
  PersistArgs a = {};
  a.n = c->n; a.nsub = c->nsub; a.n0 = c->n0; a.n_chunks = c->n0 > 0 ? c->n_chunks : 0; a.n_units = c->n_units;
  a.dots = c->flexible ? 2 : 1;
  a.rowptr = c->rowptr; a.colind = c->colind; a.dcol16 = c->dcol16; a.val = c->val;
  a.x = c->x; a.r = c->r; a.p = c->p; a.q = c->q; a.z = c->z;
  a.om_ptr = c->om_ptr; a.om_dofs = c->om_dofs; a.ainv = c->ainv; a.ainv_off = c->ainv_off;
  a.unit_ptr = c->unit_ptr; a.zloc = c->zloc;
  a.brow_ptr = c->brow_ptr; a.brow_dof = c->brow_dof; a.bcol_ptr = c->bcol_ptr; a.bcol = c->bcol;
  a.phi_off = c->phi_off; a.phi = c->phi; a.chunk_blk = c->chunk_blk; a.chunk_r0 = c->chunk_r0;
  a.chunk_r1 = c->chunk_r1; a.chunk_slot = c->chunk_slot; a.partial = c->partial;
  a.cs_ptr = c->cs_ptr; a.cs_idx = c->cs_idx;
  a.a0inv = c->fp32 ? static_cast<const void*>(c->A0inv32) : static_cast<const void*>(c->A0inv);
  a.pos_blk = c->pos_blk; a.pull_ptr = c->pull_ptr; a.pull_pos = c->pull_pos;
  a.red = c->red; a.bar = c->pbar; a.ks = c->ks; a.err = c->derr; a.wait_cycles = c->wait_cycles;
  a.max_m = c->max_m;
  a.stall_test = c->stall_test ? 1 : 0;
  void* args[] = {&a};
  if (c->fp32)
    GDSW_CK(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_pcg_persistent<float>), dim3(c->persist_grid),
                                        dim3(256), args, c->persist_smem, s));
  else
    GDSW_CK(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_pcg_persistent<double>), dim3(c->persist_grid),
                                        dim3(256), args, c->persist_smem, s));
  return GDSW_OK;
}

}  // namespace gdsw
