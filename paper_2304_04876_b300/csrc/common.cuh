// Device helpers shared by the kernels: deterministic block reductions and the
// "last CTA finishes the sum" pattern used instead of atomics on values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gdsw {

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA in a fixed tree order; the result is valid in thread 0.
// `sh` needs blockDim.x/32 entries.  Ends with a barrier so `sh` can be reused.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
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
// arrive at `ticket`; that CTA sees the partial results the others published
// before arriving (they fence first).  The ticket is reset for the next use.
__device__ __forceinline__ bool arrive_last(unsigned int* ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
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
