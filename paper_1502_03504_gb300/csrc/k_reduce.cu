// FP64 reductions over stored fields: conservation sums, the loss
// sum (u_T - target)^2 with the adjoint seed lambda_T = 2 (u_T - target), and
// the fixed-order finalisation of per-block partial sums.  Fields are stored in
// FP32/BF16 (or FP64); every sum is accumulated in FP64.
#include "device_common.cuh"

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
