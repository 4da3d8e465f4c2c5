// Calibration: the FP64 FMA rate of the device, the denominator of the FP64 kernels' ALU
// roofline.  GB300 runs FP64 far below its FP32 rate, and the FP64 Dslash, SU(3) products
// and force are bound by that pipe, not by HBM; the nominal figure (two FP64 FMAs per SM
// and clock) is replaced by this measurement.
#include "lqcd_internal.cuh"
#include "tune.cuh"

namespace {

constexpr int kChains = 16;     // independent FMA chains per thread (hide the pipe latency)
constexpr int kFmaThreads = 256;

// Each thread runs kChains independent chains a <- a * b + c for `iters` steps; the values
// stay bounded (b slightly below 1) and the sum is stored only if it is NaN, so the work
// cannot be removed and nothing is written in practice.
__global__ void __launch_bounds__(kFmaThreads) k_fma64(int iters, double b, double c, double* sink) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s != s) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" lq_status lq_fp64_fma_rate(lq_context* ctx, double* gflops) {
  if (!ctx || !gflops) return LQ_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  int per_sm = 0;
  LQ_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma64, kFmaThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const int blocks = ctx->num_sms * per_sm;
  const int iters = 1 << 13;
  void* sink = nullptr;
  lq_status st = lq_scratch(ctx, sizeof(double) * blocks, &sink);
  if (st) return st;
  cudaEvent_t e0, e1;
  LQ_CUDA(ctx, cudaEventCreate(&e0));
  LQ_CUDA(ctx, cudaEventCreate(&e1));
  float best_ms = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {   // the first run warms the clocks up; best of the rest
    cudaEventRecord(e0, 0);
    k_fma64<<<blocks, kFmaThreads>>>(iters, 0.999999999, 1e-9, (double*)sink);
    cudaEventRecord(e1, 0);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return lq_cuda_fail(ctx, e, "k_fma64");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best_ms) best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * kChains * (double)iters * kFmaThreads * blocks;
  *gflops = flops / (best_ms * 1e-3) / 1e9;
  return LQ_OK;
}
