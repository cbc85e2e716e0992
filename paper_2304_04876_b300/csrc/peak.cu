// Measured FMA throughput of the device (FP64 or FP32), the denominator of the
// arithmetic side of the rooflines: the Krylov kernels (SpMV, vector updates,
// coarse GEMV) work in FP64, whose issue rate on B300 is a small fraction of
// the FP32 one, so their bound is max(bytes / HBM bandwidth, FMAs / this rate).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gdsw {

namespace {

// Eight independent FMA chains per thread, `iters` trips; the result is
// written only under a condition the data never meets, so nothing is stored
// yet nothing can be optimised away.
template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T b, T c, T* out) {
  T a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = T(threadIdx.x + u) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int u = 0; u < 8; ++u) s += a[u];
  if (s == T(-1.2345e30)) out[blockIdx.x] = s;
}

template <class T>
gdsw_status rate_t(double* fma_per_second, cudaStream_t s) {
  int dev = 0, sms = kNumSMs, per_sm = 1;
  GDSW_CK(cudaGetDevice(&dev));
  GDSW_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GDSW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, 256, 0));
  const int grid = sms * std::max(1, per_sm);
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gdsw_status st = GDSW_OK;
  float best = 3.4e38f;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // b slightly below 1 and c small keep every chain finite
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    k_fma_chains<T><<<grid, 256, 0, s>>>(iters, T(0.999999), T(1e-7), out);   // warm-up and timed
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) k_fma_chains<T><<<grid, 256, 0, s>>>(iters, T(0.999999), T(1e-7), out);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  if (e != cudaSuccess) {
    set_error("FMA rate measurement: %s", cudaGetErrorString(e));
    st = GDSW_ERR_CUDA;
  } else {
    *fma_per_second = double(grid) * 256.0 * double(iters) * 8.0 / (double(best) * 1e-3);
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

// One random 64-bit pattern per index (splitmix64 of seed + i * golden ratio):
// as a double (every other one with its exponent moved into or near the
// binary32 range, where rounding matters) narrowed both ways, and its low 32
// bits as a float widened both ways; counts the results that differ in any bit
// (NaNs compare equal to NaNs).
__global__ void k_check_conversions(uint64_t seed, int64_t count, unsigned long long* bad) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    uint64_t x = seed + static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull;
    x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ull; x ^= x >> 27; x *= 0x94D049BB133111EBull; x ^= x >> 31;
    uint64_t y = x;
    if (i & 1) y = (x & 0x800fffffffffffffull) | (uint64_t(870 + (x >> 20) % 300) << 52);
    const double d = __longlong_as_double(static_cast<long long>(y));
    const float hw = __double2float_rn(d), sw = f32_from_f64(d);
    if (__float_as_uint(hw) != __float_as_uint(sw) && !(hw != hw && sw != sw)) atomicAdd(bad, 1ull);
    const float f = __uint_as_float(static_cast<uint32_t>(x));
    const double hd = static_cast<double>(f), sd = f64_from_f32(f);
    if (__double_as_longlong(hd) != __double_as_longlong(sd) && !(hd != hd && sd != sd)) atomicAdd(bad + 1, 1ull);
  }
}

}  // namespace

}  // namespace gdsw

extern "C" GDSW_API gdsw_status gdsw_measure_fma_rate(int32_t precision, double* fma_per_second, void* stream) {
  if (fma_per_second == nullptr || (precision != GDSW_PREC_FP64 && precision != GDSW_PREC_FP32)) {
    gdsw::set_error("gdsw_measure_fma_rate: precision must be GDSW_PREC_FP64 or GDSW_PREC_FP32 and the output non-NULL");
    return GDSW_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == GDSW_PREC_FP64 ? gdsw::rate_t<double>(fma_per_second, s)
                                : gdsw::rate_t<float>(fma_per_second, s);
}

extern "C" GDSW_API gdsw_status gdsw_check_conversions(uint64_t seed, int64_t count, uint64_t* mismatches,
                                                      void* stream) {
  if (mismatches == nullptr || count < 0) {
    gdsw::set_error("gdsw_check_conversions: mismatches must be non-NULL and count >= 0");
    return GDSW_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* bad = nullptr;
  unsigned long long host[2] = {0, 0};
  cudaError_t e = cudaMalloc(&bad, sizeof(host));
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(host), s);
  if (e == cudaSuccess && count > 0) {
    const int grid = static_cast<int>(std::min<int64_t>((count + 255) / 256, int64_t(gdsw::kNumSMs) * 16));
    gdsw::k_check_conversions<<<grid, 256, 0, s>>>(seed, count, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, bad, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (bad) cudaFree(bad);
  if (e != cudaSuccess) {
    gdsw::set_error("gdsw_check_conversions: %s", cudaGetErrorString(e));
    return GDSW_ERR_CUDA;
  }
  mismatches[0] = host[0];
  mismatches[1] = host[1];
  return GDSW_OK;
}
