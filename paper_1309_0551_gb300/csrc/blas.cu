// Vector kernels for solvers driven from outside the library (the t-split CG): y = a x + b y
// and Re<x, y> summed in FP64, on n complex values of one precision.
#include "lqcd_internal.cuh"
#include "tune.cuh"

namespace {

constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_axpby(int64_t nreal, T a, const T* __restrict__ x, T b, T* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nreal; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

// Re<x, y> = sum of x_k y_k over the reals; per-thread FP64 sums, then the deterministic block
// reduction (the last block stores the total).
template <class T>
__global__ void __launch_bounds__(kThreads) k_dot(int64_t nreal, const T* __restrict__ x, const T* __restrict__ y,
                                                  Reducer red) {
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nreal; i += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma((double)x[i], (double)y[i], acc[0]);
  block_reduce<1>(acc, red, 0, 1, blockIdx.x, gridDim.x);
}

}  // namespace

extern "C" lq_status lq_vec_axpby(lq_context* ctx, int64_t n, double a, const void* x, double b, void* y, lq_prec prec,
                                  lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (n < 0 || (prec != LQ_F64 && prec != LQ_F32)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "n >= 0, LQ_F64 or LQ_F32");
  if (n == 0) return LQ_OK;
  if (!x || !y) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "NULL vector");
  DeviceGuard dg(ctx->device);
  const int64_t nreal = 2 * n;
  int64_t blocks = (nreal + kThreads - 1) / kThreads;
  if (blocks > 8LL * ctx->num_sms) blocks = 8LL * ctx->num_sms;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == LQ_F64) k_axpby<double><<<blocks, kThreads, 0, s>>>(nreal, a, (const double*)x, b, (double*)y);
  else k_axpby<float><<<blocks, kThreads, 0, s>>>(nreal, (float)a, (const float*)x, (float)b, (float*)y);
  LQ_CHECK_LAUNCH(ctx, "k_axpby");
  return LQ_OK;
}

extern "C" lq_status lq_vec_dot(lq_context* ctx, int64_t n, const void* x, const void* y, lq_prec prec, double* result,
                                lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (n < 0 || (prec != LQ_F64 && prec != LQ_F32)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "n >= 0, LQ_F64 or LQ_F32");
  if (!x || !y || !result) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "NULL pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    LQ_CUDA(ctx, cudaMemsetAsync(result, 0, sizeof(double), s));
    return LQ_OK;
  }
  const int64_t nreal = 2 * n;
  int64_t blocks = (nreal + kThreads - 1) / kThreads;
  if (blocks > 4LL * ctx->num_sms) blocks = 4LL * ctx->num_sms;
  void* base = nullptr;
  lq_status st = lq_scratch(ctx, 256 + sizeof(double) * blocks, &base);
  if (st) return st;
  Reducer red{(double*)((char*)base + 256), (unsigned int*)base, result, (int)blocks, FIN_STORE, nullptr};
  LQ_CUDA(ctx, cudaMemsetAsync(base, 0, sizeof(unsigned int), s));
  if (prec == LQ_F64) k_dot<double><<<blocks, kThreads, 0, s>>>(nreal, (const double*)x, (const double*)y, red);
  else k_dot<float><<<blocks, kThreads, 0, s>>>(nreal, (const float*)x, (const float*)y, red);
  LQ_CHECK_LAUNCH(ctx, "k_dot");
  return LQ_OK;
}
