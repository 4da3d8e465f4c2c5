// Device guard, launch-shape autotuner and the deterministic block reduction shared by
// the kernels.
#pragma once

#include <string>
#include <type_traits>
#include <vector>

#include "lqcd_internal.cuh"

// Makes `device` current for the lifetime of the guard, restoring the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != device) {
      changed = cudaSetDevice(device) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

inline bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return true;  // be conservative
  return st != cudaStreamCaptureStatusNone;
}

// Picks a launch shape from `cands` for `key` by timing run(cand) on stream s and caches
// the choice in the context.  Each candidate is timed as kTuneBurst back-to-back launches
// (per-launch average, best of three repetitions), each burst preceded by a write of a
// buffer twice the L2 size: the first launch finds nothing in L2 and the following ones
// run the way a solver or a graph issues them, one after another.  Without tuning, or
// while the stream is being captured, the first candidate is used and nothing is cached.
constexpr int kTuneBurst = 3;
template <class F>
lq_status tune_pick(lq_context* ctx, const std::string& key, const std::vector<TuneEntry>& cands,
                    cudaStream_t s, F run, TuneEntry* pick) {
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) {
    *pick = it->second;
    return LQ_OK;
  }
  if (!ctx->tuning || cands.size() == 1 || stream_capturing(s)) {
    *pick = cands[0];
    return LQ_OK;
  }
  if (!ctx->flush) {
    size_t want = 2 * (ctx->l2_bytes ? ctx->l2_bytes : (size_t(128) << 20));
    LQ_CUDA(ctx, cudaMalloc(&ctx->flush, want));
    ctx->flush_bytes = want;
  }
  cudaEvent_t e0, e1;
  LQ_CUDA(ctx, cudaEventCreate(&e0));
  LQ_CUDA(ctx, cudaEventCreate(&e1));
  std::vector<TuneEntry> timed;
  float best_us = 1e30f;
  lq_status st = LQ_OK;
  for (const TuneEntry& c : cands) {
    st = run(c);  // warm-up (first launch of an instance loads its code)
    if (st) break;
    float us_best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaMemsetAsync(ctx->flush, rep, ctx->flush_bytes, s);
      cudaEventRecord(e0, s);
      for (int k = 0; k < kTuneBurst; ++k) run(c);
      cudaEventRecord(e1, s);
      cudaError_t err = cudaEventSynchronize(e1);
      if (err != cudaSuccess) { st = lq_cuda_fail(ctx, err, "tune"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const float us = ms * 1000.f / kTuneBurst;
      if (us < us_best) us_best = us;
    }
    if (st) break;
    TuneEntry t = c;
    t.us = us_best;
    timed.push_back(t);
    if (us_best < best_us) best_us = us_best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  // Among the shapes close to the fastest lone launch -- within 3% (timing noise) in the
  // default mode, within 15% in the throughput mode (several independent launches in
  // flight fill the GPU, so a launch's own parallelism matters less than its instruction
  // count) -- take the one doing the least redundant work: fewest threads per site, most
  // right-hand sides sharing each loaded link (per thread, or per block for the
  // rhs-per-warp kernel, which runs one thread per site and rhs), then the candidate order.
  const float tol = ctx->tune_mode == 2 ? 1.15f : 1.03f;
  auto tps_of = [](const TuneEntry& t) { return t.tps == kTpsRhsWarps || t.tps == kTpsTma || t.tps == kTpsPaired ? 1 : t.tps; };
  TuneEntry best;
  bool have = false;
  for (const TuneEntry& t : timed) {
    if (t.us > tol * best_us) continue;
    if (!have || tps_of(t) < tps_of(best) || (tps_of(t) == tps_of(best) && t.rhs_tile > best.rhs_tile)) {
      best = t;
      have = true;
    }
  }
  ctx->tune[key] = best;
  lq_tune_save(ctx);
  *pick = best;
  return LQ_OK;
}

// ------------------------------------------------------------- reductions --------------

// Per right-hand-side scalars of the conjugate-gradient iteration, device resident.
struct CGScalars {
  double rr;      // current ||r||^2 of the iterated residual
  double rr_prev; // ||r||^2 one iteration earlier (denominator of beta)
  double pAp;     // <p, M p>
  double alpha, beta;
  double alpha_last;  // alpha of the last iteration in which the system was active
  double bb;      // ||b||^2
  double tol2;    // stop threshold on rr: tol^2 * bb
  double rhi2;    // ||r||^2 of the last FP64 residual replacement
  int active;     // 1 while iterating
  int iters;      // iterations done while active
  int done;       // set by the host once the FP64 true residual met the tolerance
  int ru;         // set by the host: this system takes the reliable update now (batched solve)
};

// FIN_DEFER: the blocks only store their partials; a later kernel sums them (block_total).
// That keeps the fence, the counter atomic and the second barrier -- each an L2 round trip
// while the block still holds its SM slot -- out of a launch with many short-lived blocks.
enum { FIN_STORE = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_DEFER = 3 };

__device__ __forceinline__ void finish_one(const Reducer& red, int rhs, double total) {
  CGScalars* s = reinterpret_cast<CGScalars*>(red.finisher_state) + rhs;
  switch (red.finisher) {
    case FIN_STORE:
      red.result[rhs] = total;
      break;
    case FIN_ALPHA:
      s->pAp = total;
      s->alpha = (s->active && total > 0.0) ? s->rr / total : 0.0;
      if (s->active) s->alpha_last = s->alpha;
      break;
    case FIN_BETA:
      if (s->active) {
        s->iters += 1;
        s->rr_prev = s->rr;
        s->rr = total;
        s->beta = total / s->rr_prev;
        if (!(total > s->tol2)) s->active = 0;  // apparent convergence (or NaN)
      }
      break;
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Sum over the warp of FP32 values, returned in FP64 (valid in every lane).  A fixed xor
// shuffle tree of error-free FP32 pair sums -- Knuth's TwoSum: t = a + b rounded and
// e = (a - (t - b')) + (b - b'), b' = t - a, with t + e = a + b exactly -- keeps each
// level's rounding error in a companion term c; s + c is formed in FP64 once.  The result
// is the exact sum of the 32 values up to ~32 u^2 relative (u = 2^-24), i.e. as good as
// an FP64 tree over them, with two conversions and one FP64 add per warp instead of five
// shuffled FP64 adds: GB300's FP64 pipe runs at 1/64 of the FP32 rate, and in the CG's
// fused Dslash reduction the FP64 tree kept it a quarter busy.
__device__ __forceinline__ void warp_sum_sc(float& s, float& c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + e;
  }
}
__device__ __forceinline__ double warp_sum(float x) {
  float s = x, c = 0.f;
  warp_sum_sc(s, c);
  return (double)s + (double)c;
}

// Block-wide sum of one FP32 value per thread, in FP64 (every thread gets it): the
// compensated warp tree in each warp, the warps' (s, c) pairs through shared memory, the
// same tree over them in warp 0 -- three FP64 operations per block.  Ends with a barrier.
__device__ __forceinline__ double block_sum_f32(float x) {
  __shared__ float2 sm[32];
  __shared__ double total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float s = x, c = 0.f;
  warp_sum_sc(s, c);
  if (lane == 0) sm[warp] = make_float2(s, c);
  __syncthreads();
  if (warp == 0) {
    const float2 v = lane < nw ? sm[lane] : make_float2(0.f, 0.f);
    s = v.x;
    c = v.y;
    warp_sum_sc(s, c);
    if (lane == 0) total = (double)s + (double)c;
  }
  __syncthreads();
  return total;
}

// The block-wide helpers below (block_reduce, block_total, block_sum_store, grid_finish)
// take threadIdx.x as the thread's index in the block: they need one-dimensional blocks.
//
// Every thread of the block calls this with its NR per-rhs contributions (rhs0 + r).
// Partials go to red.partials[rhs][bx] (bx < nbx: the block's column); the last block of
// the grid to arrive sums them in column order (deterministic for a given launch shape)
// and runs the finisher, except under FIN_DEFER, where a later launch sums them.  No
// thread ever waits on another block.
// kWideFinish: the last block sums each row with all its threads (short tail; for kernels
// that finish every launch, like the CG update) or one warp per row (fewer registers for
// the whole kernel: the compiler sizes it for this rarely run path too).
// v: per-thread contributions in FP64, or in FP32 (then summed per warp by the compensated
// FP32 tree, FP64 from the warp sums up).
template <int NR, bool kWideFinish = true, class VT>
__device__ __forceinline__ void block_reduce(const VT (&v)[NR], const Reducer& red, int rhs0, int nrhs,
                                             int bx, int nbx) {
  __shared__ double sm[NR][32];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double x = warp_sum(v[r]);
    if (lane == 0) sm[r][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double x = lane < nw ? sm[r][lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0 && rhs0 + r < nrhs) red.partials[(size_t)(rhs0 + r) * nbx + bx] = x;
    }
  }
  if (red.finisher == FIN_DEFER) return;  // summed by the consumer after this launch
  __syncthreads();
  if (threadIdx.x == 0) {
    // thread 0 wrote this block's partials: make them visible before counting the block
    __threadfence();
    unsigned total = gridDim.x * gridDim.y;
    unsigned prev = atomicAdd(red.counter, 1u);
    am_last = (prev == total - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if constexpr (!kWideFinish) {
    // one warp per row, lanes strided, then a fixed shuffle tree: deterministic
    for (int rhs = warp; rhs < nrhs; rhs += nw) {
      double x = 0.0;
      for (int b = lane; b < nbx; b += 32) x += __ldcg(red.partials + (size_t)rhs * nbx + b);
      x = warp_sum(x);
      if (lane == 0) finish_one(red, rhs, x);
    }
  } else {
    // the whole block sums each row (strided by thread, then a fixed tree): deterministic
    for (int rhs = 0; rhs < nrhs; ++rhs) {
      double x = 0.0;
      for (int b = threadIdx.x; b < nbx; b += blockDim.x) x += __ldcg(red.partials + (size_t)rhs * nbx + b);
      x = warp_sum(x);
      __syncthreads();                       // sm[0][] free again
      if (lane == 0) sm[0][warp] = x;
      __syncthreads();
      if (warp == 0) {
        double y = lane < nw ? sm[0][lane] : 0.0;
        y = warp_sum(y);
        if (lane == 0) finish_one(red, rhs, y);
      }
    }
  }
  if (threadIdx.x == 0) *red.counter = 0u;
}

// Sum of row[0, n) by the whole block in a fixed order (thread-strided sums, then a fixed
// shuffle tree); every thread gets the total, the same in every block.  Reads through L2:
// the row was written by an earlier launch.
__device__ __forceinline__ double block_total(const double* row, int n) {
  __shared__ double sm[32];
  __shared__ double total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double x = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) x += __ldcg(row + b);
  x = warp_sum(x);
  if (lane == 0) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double y = lane < nw ? sm[lane] : 0.0;
    y = warp_sum(y);
    if (lane == 0) total = y;
  }
  __syncthreads();
  return total;
}

// The one-dimensional form: column = blockIdx.x of a (nbx, rhs tiles) grid.
template <int NR, class VT>
__device__ __forceinline__ void block_reduce(const VT (&v)[NR], const Reducer& red, int rhs0, int nrhs) {
  block_reduce<NR, true>(v, red, rhs0, nrhs, blockIdx.x, gridDim.x);
}

// Block-wide sums of v[r] (every thread calls); thread 0 stores sum r at dst[r * stride]
// for r < nvalid.  Ends with a barrier so shared memory can be reused by the next call.
template <int NR, class VT>
__device__ __forceinline__ void block_sum_store(const VT (&v)[NR], double* dst, size_t stride, int nvalid) {
  if constexpr (std::is_same<VT, float>::value) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double t = block_sum_f32(v[r]);
      if (threadIdx.x == 0 && r < nvalid) dst[(size_t)r * stride] = t;
    }
    return;
  }
  __shared__ double sm[NR][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double x = warp_sum(v[r]);
    if (lane == 0) sm[r][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double x = lane < nw ? sm[r][lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0 && r < nvalid) dst[(size_t)r * stride] = x;
    }
  }
  __syncthreads();
}

// Block-wide sums of v[r] added to dst[r] for r < nvalid by one thread (every thread
// calls; deterministic: a fixed tree per block, one writer).  Ends with a barrier.
template <int NR, class VT>
__device__ __forceinline__ void block_sum_add(const VT (&v)[NR], double* dst, int nvalid) {
  if constexpr (std::is_same<VT, float>::value) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double t = block_sum_f32(v[r]);
      if (threadIdx.x == 0 && r < nvalid) dst[r] += t;
    }
    return;
  }
  __shared__ double sm[NR][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double x = warp_sum(v[r]);
    if (lane == 0) sm[r][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double x = lane < nw ? sm[r][lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0 && r < nvalid) dst[r] += x;
    }
  }
  __syncthreads();
}

// End of a persistent kernel whose blocks stored per-row partials partials[q*stride + col]
// (cols(q) columns for row q): the last block to finish sums each row in column order and
// runs the finisher on it.  Every thread of every block calls this once.
template <class Cols>
__device__ __forceinline__ void grid_finish(const Reducer& red, int nq, size_t stride, Cols cols) {
  __shared__ int am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    // thread 0 wrote all of this block's partials: publish them, then count the block
    __threadfence();
    unsigned prev = atomicAdd(red.counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int q = warp; q < nq; q += nw) {
    const int n = cols(q);
    double x = 0.0;
    for (int b = lane; b < n; b += 32) x += __ldcg(red.partials + (size_t)q * stride + b);
    x = warp_sum(x);
    if (lane == 0) finish_one(red, q, x);
  }
  if (threadIdx.x == 0) *red.counter = 0u;
}
