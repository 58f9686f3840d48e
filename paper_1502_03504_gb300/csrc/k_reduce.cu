// FP64 reductions over stored fields: conservation sums, the loss
// sum (u_T - target)^2 with the adjoint seed lambda_T = 2 (u_T - target), and
// the fixed-order finalisation of per-block partial sums.  Fields are stored in
// FP32/BF16 (or FP64); every sum is accumulated in FP64.
#include <mutex>

#include "device_common.cuh"
#include "lope.h"

namespace lope {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* ws) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += ws[w];
  return s;
}

template <class T>
__global__ void __launch_bounds__(kThreads) reduce_kernel(int op, const T* __restrict__ x,
                                                           const T* __restrict__ y, int64_t n,
                                                           double* partials) {
  __shared__ double ws[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * int64_t(kThreads) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * kThreads) {
    const double a = double(to_c(x[i]));
    if (op == 0) {
      acc += a;
    } else {
      const double d = a - double(to_c(y[i]));
      acc = __fma_rn(d, d, acc);
    }
  }
  const double s = block_sum(acc, ws);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(kThreads) loss_seed_kernel(const T* __restrict__ u,
                                                              const T* __restrict__ tgt,
                                                              T* __restrict__ lam, int64_t n,
                                                              double* partials) {
  __shared__ double ws[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * int64_t(kThreads) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * kThreads) {
    const double d = double(to_c(u[i])) - double(to_c(tgt[i]));
    acc = __fma_rn(d, d, acc);
    lam[i] = from_c<T>(C_t<T>(2.0 * d));
  }
  const double s = block_sum(acc, ws);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One block sums `count` partials in a fixed order.
__global__ void __launch_bounds__(kThreads) finalize_kernel(const double* partials, int count,
                                                             double* result, int accumulate) {
  __shared__ double ws[kThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += kThreads) acc += partials[i];
  const double s = block_sum(acc, ws);
  if (threadIdx.x == 0) *result = accumulate ? *result + s : s;
}

int blocks_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  return int(b < kReduceBlocks ? b : kReduceBlocks);
}

}  // namespace

cudaError_t launch_reduce(int op, int dtype, const void* x, const void* y, int64_t n,
                          double* partials, double* result, cudaStream_t s) {
  const int b = blocks_for(n);
  switch (dtype) {
    case kF32: reduce_kernel<float><<<b, kThreads, 0, s>>>(op, (const float*)x, (const float*)y, n, partials); break;
    case kF64: reduce_kernel<double><<<b, kThreads, 0, s>>>(op, (const double*)x, (const double*)y, n, partials); break;
    case kBF16: reduce_kernel<__nv_bfloat16><<<b, kThreads, 0, s>>>(op, (const __nv_bfloat16*)x, (const __nv_bfloat16*)y, n, partials); break;
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_finalize(partials, b, result, 0, s);
}

cudaError_t launch_loss_seed(int dtype, const void* uT, const void* target, void* lam, int64_t n,
                             double* partials, double* loss, cudaStream_t s) {
  const int b = blocks_for(n);
  switch (dtype) {
    case kF32: loss_seed_kernel<float><<<b, kThreads, 0, s>>>((const float*)uT, (const float*)target, (float*)lam, n, partials); break;
    case kF64: loss_seed_kernel<double><<<b, kThreads, 0, s>>>((const double*)uT, (const double*)target, (double*)lam, n, partials); break;
    case kBF16: loss_seed_kernel<__nv_bfloat16><<<b, kThreads, 0, s>>>((const __nv_bfloat16*)uT, (const __nv_bfloat16*)target, (__nv_bfloat16*)lam, n, partials); break;
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_finalize(partials, b, loss, 0, s);
}

cudaError_t launch_finalize(const double* partials, int count, double* result, int accumulate,
                            cudaStream_t s) {
  finalize_kernel<<<1, kThreads, 0, s>>>(partials, count, result, accumulate);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lope

// ---------------------------------------------------------------------------
// Reduction that allocates nothing.
//
// Some callers cannot hand this library a scratch buffer: their device memory
// is owned entirely by another allocator (for example a framework's caching
// allocator that has reserved the whole GPU), or they run in a loop where an
// allocation call, which may synchronise the device, is not acceptable.  This
// variant of the FP64 reduction keeps its per-block partial sums in a
// file-scope device array instead.  The array is part of the library image:
// every GPU that loads the library holds its 512 KiB until the process exits.
//
// Block b sums elements [b * kNoAllocChunk, (b + 1) * kNoAllocChunk) into
// slot b, so one call needs ceil(n / kNoAllocChunk) slots and n is limited to
// kNoAllocPartials * kNoAllocChunk = 2^28 elements.  Every slot a call uses is
// written by that call before it is read, so nothing has to be cleared; the
// array keeps the last call's partial sums.  All calls on a device share the
// one array, so calls whose kernels overlap on the GPU (for example on two
// streams without ordering between them) race and must be serialised by the
// caller.
namespace lope {
namespace {

constexpr int kNoAllocPartials = 65536;
constexpr int kNoAllocPerThread = 16;
constexpr int64_t kNoAllocChunk = int64_t(kThreads) * kNoAllocPerThread;
constexpr int64_t kNoAllocMaxN = int64_t(kNoAllocPartials) * kNoAllocChunk;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

template <class T>
__global__ void __launch_bounds__(kThreads) chunk_reduce_kernel(int op, const T* __restrict__ x,
                                                                 const T* __restrict__ y,
                                                                 int64_t n, double* partials) {
  __shared__ double ws[kThreads / 32];
  const int64_t lo = int64_t(blockIdx.x) * kNoAllocChunk;
  const int64_t hi = lo + kNoAllocChunk < n ? lo + kNoAllocChunk : n;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const double a = double(to_c(x[i]));
    if (op == 0) {
      acc += a;
    } else {
      const double d = a - double(to_c(y[i]));
      acc = __fma_rn(d, d, acc);
    }
  }
  const double s = block_sum(acc, ws);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Device address of g_noalloc_partials, looked up once per device with that
// device current (host code must not pass the symbol itself to a kernel).
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};

cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lope

extern "C" lope_status lope_reduce_noalloc(int op, lope_dtype dtype, const void* x, const void* y,
                                           int64_t n, double* result_dev, void* cuda_stream) {
  using namespace lope;
  if ((op != 0 && op != 1) || !x || (op == 1 && !y) || !result_dev || n < 0)
    return lope_fail_external(LOPE_ERR_INVALID, "bad reduction argument");
  if (n > kNoAllocMaxN)
    return lope_fail_external(LOPE_ERR_INVALID,
                              "lope_reduce_noalloc: n exceeds 2^28 elements, the most its static "
                              "partial-sum array covers; use lope_reduce with a scratch buffer");
  if (dtype != LOPE_F64 && dtype != LOPE_F32 && dtype != LOPE_BF16)
    return lope_fail_external(LOPE_ERR_INVALID, "unknown dtype");
  double* partials = nullptr;
  cudaError_t e = noalloc_scratch(&partials);
  if (e != cudaSuccess) return lope_fail_external(LOPE_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = int(n == 0 ? 1 : (n + kNoAllocChunk - 1) / kNoAllocChunk);
  switch (dtype) {
    case LOPE_F32: chunk_reduce_kernel<float><<<blocks, kThreads, 0, s>>>(op, (const float*)x, (const float*)y, n, partials); break;
    case LOPE_F64: chunk_reduce_kernel<double><<<blocks, kThreads, 0, s>>>(op, (const double*)x, (const double*)y, n, partials); break;
    default: chunk_reduce_kernel<__nv_bfloat16><<<blocks, kThreads, 0, s>>>(op, (const __nv_bfloat16*)x, (const __nv_bfloat16*)y, n, partials); break;
  }
  count_launches(1);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_finalize(partials, blocks, result_dev, 0, s);
  if (e != cudaSuccess) return lope_fail_external(LOPE_ERR_CUDA, cudaGetErrorString(e));
  return LOPE_OK;
}
