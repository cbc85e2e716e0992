// gdsw_spmv_dot_noalloc: y = A x and (x, y) for callers that must not allocate
// device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand all
// device memory to their own pool allocator at start-up (a late cudaMalloc can
// then fail, or synchronise the whole device in the middle of their stream
// work), and latency-bound loops where the implicit synchronisation of an
// allocation is not acceptable.  This entry point needs no handle and no
// allocation: the caller passes the CSR matrix and the vectors in device
// memory, and the per-block partial sums of the dot product live in a
// fixed-size array compiled into the library.
//
// That array is shared by every call on a device and keeps the last call's
// contents; only the arrival counter needs to start at zero and is cleared by
// each call.  Two calls whose kernels overlap on the GPU (different streams,
// no ordering between them) race on it and give wrong dot products.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace gdsw {
namespace {

constexpr int kNoAllocThreads = 256;
// One partial sum per thread block; 65536 doubles = 512 KB held by every GPU
// that loads the library, for as long as the process lives.
constexpr int kNoAllocMaxBlocks = 65536;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];
static __device__ __align__(256) unsigned int g_noalloc_ticket[1];

// One thread block per tile of kNoAllocThreads/TPR rows (no grid-stride loop),
// TPR threads per row; block b writes its partial of (x, y) to partials[b] and
// the last block to arrive sums all partials in block order (deterministic).
template <int TPR>
__global__ void __launch_bounds__(kNoAllocThreads) k_spmv_dot_static(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colind,
    const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
    double* __restrict__ dot, double* partials, unsigned int* ticket) {
  __shared__ double sh[32];
  const int sub = threadIdx.x % TPR;
  const int row = blockIdx.x * (kNoAllocThreads / TPR) + threadIdx.x / TPR;
  double acc = 0.0;
  if (row < n) {
    const int e1 = rowptr[row + 1];
    for (int e = rowptr[row] + sub; e < e1; e += TPR) acc += val[e] * x[colind[e]];
  }
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, TPR);
  double d = 0.0;
  if (sub == 0 && row < n) {
    y[row] = acc;
    d = x[row] * acc;
  }
  const double t = block_sum(d, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (arrive_last(ticket)) {
    const double s = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) *dot = s;
  }
}

// Device addresses of the two arrays, looked up once per device.  The cache
// assumes that the device's primary context (the one the runtime API uses)
// lives as long as the process: after cudaDeviceReset the module is loaded
// again, possibly at other addresses, and the cached ones are stale, so a
// process that resets a device must not call this entry point afterwards.
struct StaticScratch {
  double* partials = nullptr;
  unsigned int* ticket = nullptr;
};
constexpr int kMaxDevices = 64;
StaticScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

gdsw_status scratch_for_current_device(StaticScratch* out) {
  int dev = 0;
  GDSW_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) { set_error("device %d out of range", dev); return GDSW_ERR_UNSUPPORTED; }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  StaticScratch& s = g_scratch[dev];
  if (s.partials == nullptr) {
    void* p = nullptr;
    void* t = nullptr;
    GDSW_CK(cudaGetSymbolAddress(&p, g_noalloc_partials));
    GDSW_CK(cudaGetSymbolAddress(&t, g_noalloc_ticket));
    s.partials = static_cast<double*>(p);
    s.ticket = static_cast<unsigned int*>(t);
  }
  *out = s;
  return GDSW_OK;
}

template <int TPR>
gdsw_status launch(int n, const int* rowptr, const int* colind, const double* val, const double* x,
                   double* y, double* dot, const StaticScratch& s, cudaStream_t st) {
  const int rows = kNoAllocThreads / TPR;
  const int64_t blocks = (int64_t(n) + rows - 1) / rows;
  if (blocks > kNoAllocMaxBlocks) {
    set_error("gdsw_spmv_dot_noalloc: n = %d needs %lld blocks of %d rows, but the static scratch "
              "holds %d partial sums (at most %lld rows at this row length)",
              n, (long long)blocks, rows, kNoAllocMaxBlocks, (long long)kNoAllocMaxBlocks * rows);
    return GDSW_ERR_UNSUPPORTED;
  }
  GDSW_CK(cudaMemsetAsync(s.ticket, 0, sizeof(unsigned int), st));
  k_spmv_dot_static<TPR><<<static_cast<int>(blocks), kNoAllocThreads, 0, st>>>(
      n, rowptr, colind, val, x, y, dot, s.partials, s.ticket);
  GDSW_CK(cudaGetLastError());
  return GDSW_OK;
}

}  // namespace
}  // namespace gdsw

using namespace gdsw;

extern "C" gdsw_status gdsw_spmv_dot_noalloc(int32_t n, int64_t nnz, const int32_t* rowptr,
                                             const int32_t* colind, const double* val,
                                             const double* x, double* y, double* dot,
                                             void* stream) {
  if (n <= 0 || nnz < 0 || !rowptr || !colind || !val || !x || !y || !dot) {
    set_error("gdsw_spmv_dot_noalloc: null pointer or non-positive n");
    return GDSW_ERR_INVALID_ARG;
  }
  const double avg = double(nnz) / n;
  const int tpr = avg <= 4.5 ? 4 : avg <= 10 ? 8 : avg <= 24 ? 16 : 32;
  const int rows = kNoAllocThreads / tpr;
  if ((int64_t(n) + rows - 1) / rows > kNoAllocMaxBlocks) {
    set_error("gdsw_spmv_dot_noalloc: n = %d exceeds the static scratch limit of %lld rows for "
              "rows of about %.0f entries", n, (long long)kNoAllocMaxBlocks * rows, avg);
    return GDSW_ERR_UNSUPPORTED;
  }
  StaticScratch s;
  gdsw_status st = scratch_for_current_device(&s);
  if (st != GDSW_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  switch (tpr) {
    case 4: return launch<4>(n, rowptr, colind, val, x, y, dot, s, cs);
    case 8: return launch<8>(n, rowptr, colind, val, x, y, dot, s, cs);
    case 16: return launch<16>(n, rowptr, colind, val, x, y, dot, s, cs);
    default: return launch<32>(n, rowptr, colind, val, x, y, dot, s, cs);
  }
}
