// Device helpers shared by the kernels: deterministic block reductions and the
// "last CTA finishes the sum" pattern used instead of atomics on values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gdsw {

// The largest shared memory a block may opt in to on this device.
inline int max_block_smem_optin() {
  static int v = -1;
  if (v < 0) {
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v = optin;
  }
  return v;
}

// The launch limit on dynamic shared memory belongs to the kernel, not to a
// handle, so every opt-in kernel is raised once to the most it can take (the
// opt-in maximum less its static shared memory) and each launch asks for what
// it needs: handles with different needs then never conflict.
template <class K>
cudaError_t allow_max_dynamic_smem(K* kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_block_smem_optin() - static_cast<int>(fa.sharedSizeBytes));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---- FP64 <-> FP32 conversions on the integer ALUs ----------------------
// On B300 the hardware conversions between double and float issue on the FP64
// pipe (one warp instruction per 16 SM cycles, shared with every DFMA).  These
// two convert normal numbers by rewriting the IEEE 754 binary64 / binary32
// fields (exponent bias 1023 vs 127, 52 vs 23 fraction bits) with integer
// operations; zeros take a direct path and only subnormals, infinities and
// NaNs go to the hardware conversion.  The narrowing rounds to nearest, ties
// to even (the default IEEE 754 rounding): the dropped 29 fraction bits are
// compared with one half ulp, a carry out of the fraction correctly bumps the
// exponent and, at the top of the range, produces the infinity that rounding
// gives.  Both are checked bit for bit against the hardware conversion over
// random bit patterns (gdsw_check_conversions).
static __device__ __noinline__ float f32_from_f64_hw(double d) { return __double2float_rn(d); }
static __device__ __noinline__ double f64_from_f32_hw(float f) { return static_cast<double>(f); }

// From the binary64 bit pattern (callers that load the bits directly keep the
// compiler from handling the value as a double at all).
__device__ __forceinline__ float f32_from_f64_bits(uint64_t u) {
  const uint64_t a = u & 0x7fffffffffffffffull;
  const uint32_t sign = static_cast<uint32_t>(u >> 32) & 0x80000000u;
  // binary64 exponents 897..1150 are the binary32 normal exponents 1..254
  if (a - (uint64_t(897) << 52) < (uint64_t(1151 - 897) << 52)) {
    const uint64_t t = a - (uint64_t(896) << 52);
    uint32_t f = static_cast<uint32_t>(t >> 29);
    const uint32_t rem = static_cast<uint32_t>(t) & 0x1fffffffu;
    f += (rem > 0x10000000u) | ((rem == 0x10000000u) & f);
    return __uint_as_float(f | sign);
  }
  if (a == 0) return __uint_as_float(sign);
  return f32_from_f64_hw(__longlong_as_double(static_cast<long long>(u)));
}

__device__ __forceinline__ float f32_from_f64(double d) {
  return f32_from_f64_bits(static_cast<uint64_t>(__double_as_longlong(d)));
}

__device__ __forceinline__ double f64_from_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  const uint64_t sign = static_cast<uint64_t>(u & 0x80000000u) << 32;
  if (a - 0x00800000u < 0x7f000000u)   // normal: exponent 1..254
    return __longlong_as_double(static_cast<long long>(((static_cast<uint64_t>(a) << 29) + (uint64_t(896) << 52)) | sign));
  if (a == 0) return __longlong_as_double(static_cast<long long>(sign));
  return f64_from_f32_hw(f);
}

// Narrowing of an FP64 vector entry to the apply's compute type.
template <class T>
__device__ __forceinline__ T narrow(double d) { return static_cast<T>(d); }
template <>
__device__ __forceinline__ float narrow<float>(double d) { return f32_from_f64(d); }

// An FP64 vector entry as its bit pattern, and a bit pattern narrowed to T.
// Gathers load every entry's bits first and convert afterwards: the
// conversion's rare hardware branch would otherwise keep the compiler from
// issuing the later loads before the earlier conversions.
__device__ __forceinline__ uint64_t load_bits(const double* __restrict__ x, int i) {
  return reinterpret_cast<const unsigned long long*>(x)[i];
}
template <class T>
__device__ __forceinline__ T narrow_bits(uint64_t u) { return __longlong_as_double(static_cast<long long>(u)); }
template <>
__device__ __forceinline__ float narrow_bits<float>(uint64_t u) { return f32_from_f64_bits(u); }

// Widening of a compute-type value to FP64.
template <class T>
__device__ __forceinline__ double widen(T v) { return static_cast<double>(v); }
template <>
__device__ __forceinline__ double widen<float>(float v) { return f64_from_f32(v); }

// Sum over the CTA in a fixed order; the result is valid in thread 0.  `sh`
// needs blockDim.x/32 entries.  Ends with a barrier so `sh` can be reused.
// B300's FP64 pipe issues one warp instruction per 16 SM cycles however few
// lanes are active, so for doubles in CTAs of up to 256 threads the values are
// parked in shared memory and summed by one warp (lane l adds the l-th value of
// each warp in ascending warp order, then a shuffle tree): 8 + 5 FP64
// instructions per CTA instead of a shuffle tree in every warp (45).
template <class T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (sizeof(T) == 8 && blockDim.x <= 256) {
    __shared__ T park[256];
    park[threadIdx.x] = v;
    __syncthreads();
    T s = T(0);
    if (w == 0) {
      s = lane < int(blockDim.x) ? park[lane] : T(0);
      for (int q = 1; q < nw; ++q) {
        const int i = q * 32 + lane;
        if (i < int(blockDim.x)) s += park[i];
      }
      s = warp_sum(s);
    }
    __syncthreads();
    return s;
  }
  v = warp_sum(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    s = (lane < nw) ? sh[lane] : T(0);
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

// Returns true in every thread of the CTA that is the last of the grid to
// arrive at `ticket`.  Thread 0 must have published the CTA's partial result
// before the call; it fences that write, so the last CTA sees every partial.
// The ticket is reset for the next use.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x * gridDim.y - 1);
    if (last) *ticket = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of `count` partials in index order by one CTA (deterministic).
__device__ __forceinline__ double sum_partials(const double* part, int count, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += __ldcg(part + i);
  return block_sum(v, sh);
}

}  // namespace gdsw

namespace gdsw {

// ---- TMA bulk copies and mbarriers (sm_90+ PTX) ---------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Per-thread asynchronous copies global -> shared (sm_80+ cp.async): 16 bytes
// (L2 only) or 8 bytes, both addresses aligned to the size; the issuing thread
// sees the data after the wait on its group, other threads after a barrier.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (release at CTA scope) on a barrier whose expected count is 1.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Prefetch of a global range into L2 (no completion to wait for); src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false when `cycles` SM clock cycles (about 1 s for 2e9)
// passed without the phase completing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > cycles) return false;
  return true;
}

}  // namespace gdsw
