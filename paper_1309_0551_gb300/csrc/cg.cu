// Conjugate gradient on M = m^2 - D_eo D_oe (even sites): plain FP64, and mixed precision
// with FP64 reliable updates.
//
// One inner iteration is four kernels on the library's work stream:
//   xpay    p = r + beta p                      (skipped for inactive right-hand sides)
//   dslash  t = D_oe p                          (odd sites)
//   dslash  Ap = m^2 p - D_eo t, pAp = <p, Ap>  (fused epilogue; last block forms alpha)
//   update  x += alpha p, r -= alpha Ap, rr = ||r||^2 (last block forms beta, stop flag)
// All scalars stay on the device.  `check_every` iterations are captured once as a CUDA
// graph and replayed; between replays the host reads the per-rhs scalars (one small
// device-to-host copy) and decides on reliable updates and termination.
//
// Reliable update (mixed precision, and the FP64 solver's restart on apparent
// convergence): x_hi += x_lo, r_hi = b - M_fp64 x_hi (two FP64 half Dslash, the second with
// a fused ||r_hi||^2), r_lo = r_hi rounded, x_lo = 0, p kept, beta = ||r_lo||^2 / rr_prev.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "lqcd_internal.cuh"
#include "tune.cuh"

bool dslash_vec_ok(lq_prec gauge, lq_prec vec);

namespace {

constexpr int kBlas = 256;  // threads per block of the vector kernels

template <class T> __device__ __forceinline__ double site_norm2(const T* v) {
  T s = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) s = fma(v[k], v[k], s);
  return (double)s;
}

// x += alpha p; r -= alpha Ap; ||r||^2 -> FIN_BETA.  grid = (nbx, nrhs).
template <lq_prec VP>
__global__ void __launch_bounds__(kBlas) k_cg_update(void* x, void* r, const void* p, const void* Ap,
                                                     int Vh, Reducer red) {
  using VT = VecT<VP>;
  using T = typename VT::real;
  const int rhs = blockIdx.y;
  const CGScalars* sc = reinterpret_cast<const CGScalars*>(red.finisher_state) + rhs;
  const T alpha = (T)sc->alpha;
  double acc[1] = {0.0};
  const size_t off = (size_t)rhs * Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    T xv[6], rv[6], pv[6], av[6];
    VT::load_rw(x, off + i, xv);
    VT::load_rw(r, off + i, rv);
    VT::load(p, off + i, pv);
    VT::load(Ap, off + i, av);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      xv[k] = fma(alpha, pv[k], xv[k]);
      rv[k] = fma(-alpha, av[k], rv[k]);
    }
    VT::store(x, off + i, xv);
    VT::store(r, off + i, rv);
    acc[0] += site_norm2(rv);
  }
  block_reduce<1>(acc, red, rhs, gridDim.y);
}

// p = r + beta p for active right-hand sides.  grid = (nbx, nrhs).
template <lq_prec VP>
__global__ void __launch_bounds__(kBlas) k_cg_xpay(const void* r, void* p, const CGScalars* sc, int Vh) {
  using VT = VecT<VP>;
  using T = typename VT::real;
  const int rhs = blockIdx.y;
  if (!sc[rhs].active) return;
  const T beta = (T)sc[rhs].beta;
  const size_t off = (size_t)rhs * Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    T rv[6], pv[6];
    VT::load(r, off + i, rv);
    VT::load_rw(p, off + i, pv);
#pragma unroll
    for (int k = 0; k < 6; ++k) pv[k] = fma(beta, pv[k], rv[k]);
    VT::store(p, off + i, pv);
  }
}

// dst (precision VD) = src (precision VS) for every rhs; optional ||dst||^2 -> FIN_STORE.
template <lq_prec VS, lq_prec VD>
__global__ void __launch_bounds__(kBlas) k_convert(const void* src, void* dst, int Vh, int reduce, Reducer red) {
  using S = VecT<VS>;
  using D = VecT<VD>;
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * Vh;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    typename S::real a[6];
    typename D::real b[6];
    S::load(src, off + i, a);
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k] = (typename D::real)a[k];
    D::store(dst, off + i, b);
    if (reduce) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += (double)b[k] * (double)b[k];
      acc[0] += s;
    }
  }
  if (reduce) block_reduce<1>(acc, red, rhs, gridDim.y);
}

// x_hi += x_lo; x_lo = 0.
template <lq_prec VL>
__global__ void __launch_bounds__(kBlas) k_fold(double* x_hi, void* x_lo, int Vh) {
  using L = VecT<VL>;
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * Vh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    typename L::real a[6], z[6];
    double h[6];
    L::load_rw(x_lo, off + i, a);
    VecT<LQ_F64>::load_rw(x_hi, off + i, h);
#pragma unroll
    for (int k = 0; k < 6; ++k) { h[k] += (double)a[k]; z[k] = 0; }
    VecT<LQ_F64>::store(x_hi, off + i, h);
    L::store(x_lo, off + i, z);
  }
}

// Bump allocator over the context's scratch space.
struct Arena {
  char* base;
  size_t off = 0;
  void* take(size_t bytes) {
    off = (off + 255) / 256 * 256;
    void* p = base + off;
    off += bytes;
    return p;
  }
};

struct Solver {
  lq_context* ctx;
  cudaStream_t s;
  const lq_gauge* Uhi;
  const lq_gauge* Ulo;   // == Uhi for the plain FP64 solve
  lq_prec vp;            // inner vector precision
  bool mixed;
  double mass;
  int nrhs, Vh, nbx;
  const double* b;
  double* x;             // user solution (FP64)
  // inner vectors (precision vp)
  void *xl, *r, *p, *Ap, *t;
  // FP64 work vectors
  double *rhi, *thi;
  CGScalars* sc;         // device
  CGScalars* sc_host;    // pinned
  double* result;        // device [nrhs]
  double* partials;
  unsigned int* counter;
  int nblocks_max;

  Reducer reducer(int fin) const {
    return Reducer{partials, counter, result, nblocks_max, fin, (void*)sc};
  }
  size_t vbytes(lq_prec q) const { return (size_t)nrhs * Vh * 6 * lq_prec_bytes(q); }
};

lq_status launch_blas_update(Solver& S) {
  dim3 grid(S.nbx, S.nrhs);
  Reducer red = S.reducer(FIN_BETA);
  if (S.vp == LQ_F64) k_cg_update<LQ_F64><<<grid, kBlas, 0, S.s>>>(S.xl, S.r, S.p, S.Ap, S.Vh, red);
  else k_cg_update<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.xl, S.r, S.p, S.Ap, S.Vh, red);
  LQ_CHECK_LAUNCH(S.ctx, "k_cg_update");
  return LQ_OK;
}

lq_status launch_xpay(Solver& S) {
  dim3 grid(S.nbx, S.nrhs);
  if (S.vp == LQ_F64) k_cg_xpay<LQ_F64><<<grid, kBlas, 0, S.s>>>(S.r, S.p, S.sc, S.Vh);
  else k_cg_xpay<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.r, S.p, S.sc, S.Vh);
  LQ_CHECK_LAUNCH(S.ctx, "k_cg_xpay");
  return LQ_OK;
}

// One inner iteration.
lq_status iteration(Solver& S) {
  lq_status st = launch_xpay(S);
  if (st) return st;
  DslashArgs d;
  d.U = S.Ulo;
  d.in = S.p;
  d.out = S.t;
  d.out_parity = 1;
  d.nrhs = S.nrhs;
  d.vec_prec = S.vp;
  d.rhs_stride = S.Vh;
  st = launch_dslash(S.ctx, d, S.s);
  if (st) return st;
  Reducer red = S.reducer(FIN_ALPHA);
  DslashArgs e = d;
  e.in = S.t;
  e.out = S.Ap;
  e.out_parity = 0;
  e.w1 = S.p;
  e.a1 = S.mass * S.mass;
  e.c = -1.0;
  e.reduce = RED_DOT;
  e.red = &red;
  st = launch_dslash(S.ctx, e, S.s);
  if (st) return st;
  return launch_blas_update(S);
}

// r_hi = b - M x_hi in FP64 and ||r_hi||^2 -> result (FIN_STORE).
lq_status true_residual(Solver& S) {
  DslashArgs d;
  d.U = S.Uhi;
  d.in = S.x;
  d.out = S.thi;
  d.out_parity = 1;
  d.nrhs = S.nrhs;
  d.vec_prec = LQ_F64;
  d.rhs_stride = S.Vh;
  lq_status st = launch_dslash(S.ctx, d, S.s);
  if (st) return st;
  Reducer red = S.reducer(FIN_STORE);
  DslashArgs e = d;
  e.in = S.thi;
  e.out = S.rhi;
  e.out_parity = 0;
  e.w1 = S.b;
  e.a1 = 1.0;
  e.w2 = S.x;
  e.a2 = -S.mass * S.mass;
  e.c = 1.0;
  e.reduce = RED_NORM;
  e.red = &red;
  return launch_dslash(S.ctx, e, S.s);
}

lq_status fold_x(Solver& S) {
  if (!S.mixed) return LQ_OK;  // the FP64 solve iterates on x itself
  dim3 grid(S.nbx, S.nrhs);
  k_fold<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.x, S.xl, S.Vh);
  LQ_CHECK_LAUNCH(S.ctx, "k_fold");
  return LQ_OK;
}

// r_lo = round(r_hi) with ||r_lo||^2 -> result.
lq_status replace_residual(Solver& S) {
  dim3 grid(S.nbx, S.nrhs);
  Reducer red = S.reducer(FIN_STORE);
  if (S.mixed) k_convert<LQ_F64, LQ_F32><<<grid, kBlas, 0, S.s>>>(S.rhi, S.r, S.Vh, 1, red);
  else k_convert<LQ_F64, LQ_F64><<<grid, kBlas, 0, S.s>>>(S.rhi, S.r, S.Vh, 1, red);
  LQ_CHECK_LAUNCH(S.ctx, "k_convert");
  return LQ_OK;
}

lq_status sync_scalars(Solver& S) {
  LQ_CUDA(S.ctx, cudaMemcpyAsync(S.sc_host, S.sc, sizeof(CGScalars) * S.nrhs, cudaMemcpyDeviceToHost, S.s));
  LQ_CUDA(S.ctx, cudaStreamSynchronize(S.s));
  return LQ_OK;
}

lq_status push_scalars(Solver& S) {
  LQ_CUDA(S.ctx, cudaMemcpyAsync(S.sc, S.sc_host, sizeof(CGScalars) * S.nrhs, cudaMemcpyHostToDevice, S.s));
  return LQ_OK;
}

lq_status read_result(Solver& S, std::vector<double>& out) {
  out.resize(S.nrhs);
  LQ_CUDA(S.ctx, cudaMemcpyAsync(out.data(), S.result, sizeof(double) * S.nrhs, cudaMemcpyDeviceToHost, S.s));
  LQ_CUDA(S.ctx, cudaStreamSynchronize(S.s));
  return LQ_OK;
}

lq_status work_stream(lq_context* ctx, cudaStream_t* out) {
  static thread_local cudaStream_t cache[64] = {};
  int dev = ctx->device;
  if (dev < 0 || dev >= 64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "device index");
  if (!cache[dev]) LQ_CUDA(ctx, cudaStreamCreateWithFlags(&cache[dev], cudaStreamNonBlocking));
  *out = cache[dev];
  return LQ_OK;
}

struct GraphHolder {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  ~GraphHolder() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
  }
};

lq_status run_solver(Solver& S, const lq_cg_params& P, lq_cg_stats* stats, int* converged_all,
                     bool use_graph = true) {
  lq_context* ctx = S.ctx;
  const int n = S.nrhs;
  const double tol2 = P.tol * P.tol;
  std::vector<double> res;
  std::vector<int> done(n, 0), updates(n, 0), frozen_iters(n, 0);
  std::vector<double> bb(n);
  lq_status st;

  // ---- initial state: x = 0, r = p = 0, r_hi = b, r = round(b), rr = ||r||^2
  LQ_CUDA(ctx, cudaMemsetAsync(S.x, 0, S.vbytes(LQ_F64), S.s));
  if (S.mixed) LQ_CUDA(ctx, cudaMemsetAsync(S.xl, 0, S.vbytes(S.vp), S.s));
  LQ_CUDA(ctx, cudaMemsetAsync(S.p, 0, S.vbytes(S.vp), S.s));
  {
    dim3 grid(S.nbx, n);
    Reducer red = S.reducer(FIN_STORE);
    k_convert<LQ_F64, LQ_F64><<<grid, kBlas, 0, S.s>>>(S.b, S.rhi, S.Vh, 1, red);
    LQ_CHECK_LAUNCH(ctx, "k_convert(b)");
    st = read_result(S, res);
    if (st) return st;
  }
  for (int i = 0; i < n; ++i) {
    bb[i] = res[i];
    if (!isfinite(bb[i])) return lq_fail(ctx, LQ_ERR_NUMERIC, "source %d holds NaN/Inf", i);
  }
  st = replace_residual(S);
  if (st) return st;
  st = read_result(S, res);
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    CGScalars& c = S.sc_host[i];
    memset(&c, 0, sizeof c);
    c.rr = res[i];
    c.bb = bb[i];
    c.tol2 = tol2 * bb[i];
    c.rhi2 = bb[i];
    c.beta = 0.0;           // first xpay: p = r
    c.active = bb[i] > 0.0;
    if (bb[i] == 0.0) done[i] = 1;  // x = 0 solves it exactly
  }
  st = push_scalars(S);
  if (st) return st;

  GraphHolder graph;
  const int block = P.check_every > 0 ? P.check_every : 20;
  int total = 0, since = 0, restarts_left = 8;
  bool first = true;
  while (true) {
    bool any_active = false;
    for (int i = 0; i < n; ++i) any_active |= S.sc_host[i].active != 0;
    if (!any_active) {
      bool all_done = true;
      for (int i = 0; i < n; ++i) all_done &= done[i] != 0;
      if (all_done) break;
    }
    if (total >= P.maxiter) break;
    if (any_active) {
      // ---- a block of inner iterations
      if (first || !use_graph) {
        for (int k = 0; k < block; ++k) {
          st = iteration(S);
          if (st) return st;
        }
        first = false;
      } else {
        if (!graph.e) {
          LQ_CUDA(ctx, cudaStreamBeginCapture(S.s, cudaStreamCaptureModeThreadLocal));
          lq_status cst = LQ_OK;
          for (int k = 0; k < block && !cst; ++k) cst = iteration(S);
          cudaError_t ce = cudaStreamEndCapture(S.s, &graph.g);
          if (cst) return cst;
          LQ_CUDA(ctx, ce);
          LQ_CUDA(ctx, cudaGraphInstantiate(&graph.e, graph.g, 0));
        }
        LQ_CUDA(ctx, cudaGraphLaunch(graph.e, S.s));
      }
      total += block;
      since += block;
      st = sync_scalars(S);
      if (st) return st;
    }
    // ---- decide on a reliable update
    bool need = false;
    for (int i = 0; i < n; ++i) {
      const CGScalars& c = S.sc_host[i];
      if (!isfinite(c.rr)) return lq_fail(ctx, LQ_ERR_NUMERIC, "residual of rhs %d became NaN/Inf", i);
      if (done[i]) continue;
      if (!c.active) need = true;  // apparent convergence: verify in FP64
      if (S.mixed && (since >= P.reliable_every || c.rr < P.delta * P.delta * c.rhi2)) need = true;
    }
    if (!need) continue;
    st = fold_x(S);
    if (st) return st;
    st = true_residual(S);
    if (st) return st;
    std::vector<double> rhi2;
    st = read_result(S, rhi2);
    if (st) return st;
    st = replace_residual(S);
    if (st) return st;
    std::vector<double> rlo2;
    st = read_result(S, rlo2);
    if (st) return st;
    since = 0;
    bool restarted = false;
    for (int i = 0; i < n; ++i) {
      CGScalars& c = S.sc_host[i];
      if (done[i]) { c.active = 0; continue; }
      updates[i] += 1;
      if (!isfinite(rhi2[i])) return lq_fail(ctx, LQ_ERR_NUMERIC, "true residual of rhs %d is NaN/Inf", i);
      if (rhi2[i] <= tol2 * bb[i]) {
        done[i] = 1;
        c.active = 0;
        frozen_iters[i] = c.iters;
        continue;
      }
      if (!c.active) restarted = true;
      c.rhi2 = rhi2[i];
      c.beta = c.rr_prev > 0.0 ? rlo2[i] / c.rr_prev : 0.0;
      c.rr = rlo2[i];
      c.active = 1;
    }
    if (restarted && !S.mixed && --restarts_left < 0) break;
    st = push_scalars(S);
    if (st) return st;
  }
  // ---- final true residuals
  st = fold_x(S);
  if (st) return st;
  st = true_residual(S);
  if (st) return st;
  st = read_result(S, res);
  if (st) return st;
  int all = 1;
  for (int i = 0; i < n; ++i) {
    double rel = bb[i] > 0 ? sqrt(res[i] / bb[i]) : 0.0;
    if (!(rel <= P.tol)) all = 0;
    if (stats) {
      stats[i].iters = S.sc_host[i].iters;
      stats[i].reliable_updates = updates[i];
      stats[i].true_rel_resid = rel;
    }
  }
  *converged_all = all;
  return LQ_OK;
}

}  // namespace

extern "C" lq_status cg_solve(lq_context* ctx, const lq_gauge* U_hi, const lq_gauge* U_lo, double mass,
                              const void* b, void* x, int nrhs, const lq_cg_params* params,
                              lq_cg_stats* stats, lq_stream stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U_hi || !params) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_hi and params are required");
  if (U_hi->prec != LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_hi must be an LQ_F64 gauge");
  if (U_lo) {
    if (U_lo->prec == LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_lo must be LQ_F32, LQ_BF16 or LQ_F16");
    for (int i = 0; i < 4; ++i)
      if (U_lo->dims[i] != U_hi->dims[i]) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_lo and U_hi lattices differ");
  }
  if (!b || !x || !lq_aligned16(b) || !lq_aligned16(x))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "b and x must be non-NULL 16-byte aligned device pointers");
  if (b == x) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "b and x must be distinct");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (!(params->tol > 0.0) || params->maxiter < 1 || params->check_every < 1 || params->reliable_every < 1 ||
      !(params->delta >= 0.0 && params->delta < 1.0))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "bad CG parameters");
  DeviceGuard dg(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->mu);

  Solver S{};
  S.ctx = ctx;
  S.Uhi = U_hi;
  S.Ulo = U_lo ? U_lo : U_hi;
  S.mixed = U_lo != nullptr;
  S.vp = S.mixed ? LQ_F32 : LQ_F64;
  S.mass = mass;
  S.nrhs = nrhs;
  S.Vh = U_hi->Vh;
  S.b = (const double*)b;
  S.x = (double*)x;
  S.nbx = (S.Vh + kBlas - 1) / kBlas;
  if (S.nbx > 8 * ctx->num_sms) S.nbx = 8 * ctx->num_sms;
  S.nblocks_max = (S.Vh + 15) / 16;  // Dslash reductions: up to 4 threads per site, blocks of 64
  if (S.nblocks_max < S.nbx) S.nblocks_max = S.nbx;

  const size_t vin = S.vbytes(S.vp), v64 = S.vbytes(LQ_F64);
  const size_t need = 5 * vin + 2 * v64 + nrhs * (sizeof(CGScalars) + 8) + 8 +
                      (size_t)nrhs * S.nblocks_max * sizeof(double) + 12 * 256;
  void* base = nullptr;
  lq_status st = lq_scratch(ctx, need, &base);
  if (st) return st;
  Arena A{(char*)base};
  S.xl = S.mixed ? A.take(vin) : x;
  S.r = A.take(vin);
  S.p = A.take(vin);
  S.Ap = A.take(vin);
  S.t = A.take(vin);
  S.rhi = (double*)A.take(v64);
  S.thi = (double*)A.take(v64);
  S.sc = (CGScalars*)A.take(sizeof(CGScalars) * nrhs);
  S.result = (double*)A.take(sizeof(double) * nrhs);
  S.counter = (unsigned int*)A.take(sizeof(unsigned int));
  S.partials = (double*)A.take(sizeof(double) * nrhs * S.nblocks_max);
  if (A.off > need) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "internal: scratch layout overflow");
  if (ctx->host_pinned_bytes < sizeof(CGScalars) * nrhs) {
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    LQ_CUDA(ctx, cudaMallocHost(&ctx->host_pinned, 16 * sizeof(CGScalars)));
    ctx->host_pinned_bytes = 16 * sizeof(CGScalars);
  }
  S.sc_host = (CGScalars*)ctx->host_pinned;

  // Run on the library's own stream (capturable), ordered after the caller's stream.
  cudaStream_t user = (cudaStream_t)stream;
  st = work_stream(ctx, &S.s);
  if (st) return st;
  cudaEvent_t ev;
  LQ_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  LQ_CUDA(ctx, cudaEventRecord(ev, user));
  LQ_CUDA(ctx, cudaStreamWaitEvent(S.s, ev, 0));
  LQ_CUDA(ctx, cudaMemsetAsync(S.counter, 0, sizeof(unsigned int), S.s));
  int converged = 0;
  st = run_solver(S, *params, stats, &converged);
  cudaEventRecord(ev, S.s);
  cudaStreamWaitEvent(user, ev, 0);
  cudaEventDestroy(ev);
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < nrhs; ++i) stats[i].seconds = secs;
  if (st) return st;
  if (!converged) return lq_fail(ctx, LQ_ERR_NOT_CONVERGED, "CG did not reach tol %.3g within %d iterations",
                                 params->tol, params->maxiter);
  return LQ_OK;
}

// ------------------------------------------------------------- allocation-free solve ---
//
// Some callers may not allocate GPU memory at the point where they solve: code running
// under a caller-managed memory pool or budget, plugins whose host framework forbids
// cudaMalloc/cudaFree on its worker threads, or loops that must not synchronise the
// device the way cudaMalloc/cudaFree can.  cg_solve_noalloc serves them: it runs the same
// solver as cg_solve, but its scratch space (work vectors, per-rhs scalars, reduction
// partials) lives in the fixed array below, and it creates no stream, event or graph.
// The array is part of the library image: every GPU that loads the library holds these
// bytes until the process exits.

static constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_cg_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {};

// Device address of the static array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device with
// cudaGetSymbolAddress (which needs that device current) and cached.
static lq_status noalloc_scratch(lq_context* ctx, void** out) {
  const int dev = ctx->device;
  if (dev < 0 || dev >= 64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cg_noalloc_scratch);
    if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "cudaGetSymbolAddress(g_cg_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return LQ_OK;
}

extern "C" lq_status cg_solve_noalloc(lq_context* ctx, const lq_gauge* U_hi, const lq_gauge* U_lo, double mass,
                                      const void* b, void* x, int nrhs, const lq_cg_params* params,
                                      lq_cg_stats* stats, lq_stream stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U_hi || !params) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_hi and params are required");
  if (U_hi->prec != LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_hi must be an LQ_F64 gauge");
  if (U_lo) {
    if (U_lo->prec == LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_lo must be LQ_F32, LQ_BF16 or LQ_F16");
    for (int i = 0; i < 4; ++i)
      if (U_lo->dims[i] != U_hi->dims[i]) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_lo and U_hi lattices differ");
  }
  if (!b || !x || !lq_aligned16(b) || !lq_aligned16(x))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "b and x must be non-NULL 16-byte aligned device pointers");
  if (b == x) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "b and x must be distinct");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (!(params->tol > 0.0) || params->maxiter < 1 || params->check_every < 1 || params->reliable_every < 1 ||
      !(params->delta >= 0.0 && params->delta < 1.0))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "bad CG parameters");
  DeviceGuard dg(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->mu);

  Solver S{};
  S.ctx = ctx;
  S.Uhi = U_hi;
  S.Ulo = U_lo ? U_lo : U_hi;
  S.mixed = U_lo != nullptr;
  S.vp = S.mixed ? LQ_F32 : LQ_F64;
  S.mass = mass;
  S.nrhs = nrhs;
  S.Vh = U_hi->Vh;
  S.b = (const double*)b;
  S.x = (double*)x;
  S.nbx = (S.Vh + kBlas - 1) / kBlas;
  if (S.nbx > 8 * ctx->num_sms) S.nbx = 8 * ctx->num_sms;
  S.nblocks_max = (S.Vh + 15) / 16;  // Dslash reductions: up to 4 threads per site, blocks of 64
  if (S.nblocks_max < S.nbx) S.nblocks_max = S.nbx;
  const size_t vin = S.vbytes(S.vp), v64 = S.vbytes(LQ_F64);
  const size_t need = (S.mixed ? 5 : 4) * vin + 2 * v64 + nrhs * (sizeof(CGScalars) + 8) + 8 +
                      (size_t)nrhs * S.nblocks_max * sizeof(double) + 12 * 256;
  if (need > kNoAllocScratchBytes)
    return lq_fail(ctx, LQ_ERR_INVALID_ARG,
                   "cg_solve_noalloc: %d right-hand sides on %d sites per parity need %zu bytes of scratch, "
                   "more than its fixed %zu-byte array; use cg_solve", nrhs, S.Vh, need, kNoAllocScratchBytes);
  void* base = nullptr;
  lq_status st = noalloc_scratch(ctx, &base);
  if (st) return st;
  Arena A{(char*)base};
  S.xl = S.mixed ? A.take(vin) : x;
  S.r = A.take(vin);
  S.p = A.take(vin);
  S.Ap = A.take(vin);
  S.t = A.take(vin);
  S.rhi = (double*)A.take(v64);
  S.thi = (double*)A.take(v64);
  S.sc = (CGScalars*)A.take(sizeof(CGScalars) * nrhs);
  S.result = (double*)A.take(sizeof(double) * nrhs);
  S.counter = (unsigned int*)A.take(sizeof(unsigned int));
  S.partials = (double*)A.take(sizeof(double) * nrhs * S.nblocks_max);
  if (A.off > kNoAllocScratchBytes) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "internal: scratch layout overflow");
  CGScalars host_scalars[16];  // pageable host copy of the per-rhs scalars
  S.sc_host = host_scalars;
  S.s = (cudaStream_t)stream;  // the caller's stream: nothing is created

  // The array keeps the previous call's contents; the reduction counter must start at 0
  // (every other scratch word is written before it is read).
  LQ_CUDA(ctx, cudaMemsetAsync(S.counter, 0, sizeof(unsigned int), S.s));
  // Launch shapes come from the context's tuning table when an earlier call tuned them,
  // else the defaults: no timing runs here.
  const bool tuning = ctx->tuning;
  ctx->tuning = false;
  int converged = 0;
  st = run_solver(S, *params, stats, &converged, /*use_graph=*/false);
  ctx->tuning = tuning;
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < nrhs; ++i) stats[i].seconds = secs;
  if (st) return st;
  if (!converged) return lq_fail(ctx, LQ_ERR_NOT_CONVERGED, "CG did not reach tol %.3g within %d iterations",
                                 params->tol, params->maxiter);
  return LQ_OK;
}
