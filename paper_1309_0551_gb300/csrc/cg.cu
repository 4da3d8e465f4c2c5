// Conjugate gradient on M = m^2 - D_eo D_oe (even sites): plain FP64, and mixed precision
// with FP64 reliable updates.
//
// One inner iteration is five kernels on the library's work stream:
//   xpay    p = r + beta p                      (skipped for inactive right-hand sides)
//   dslash  t = D_oe p                          (odd sites)
//   dslash  Ap = m^2 p - D_eo t, <p, Ap>        (fused epilogue; per-block partials only)
//   pap     <p,Ap> group sums                   (32 blocks per rhs over the partials)
//   update  alpha = rr / <p,Ap> in every block, x += alpha p, r -= alpha Ap,
//           rr = ||r||^2 (last block forms beta, stop flag)
// (The batched solve forms alpha with k_cg_alpha, one block per system, instead.)
// All scalars stay on the device.  `check_every` iterations are captured once as a CUDA
// graph and replayed; between replays the host reads the per-rhs scalars (one small
// device-to-host copy) and decides on reliable updates and termination.
//
// Reliable update (mixed precision, and the FP64 solver's restart on apparent
// convergence): x_hi += x_lo, r_hi = b - M_fp64 x_hi (two FP64 half Dslash, the second with
// a fused ||r_hi||^2), r_lo = r_hi rounded, x_lo = 0, p kept, and beta in the Polak-Ribiere
// form max(0, Re<r_lo, r_lo - r_k>) / ||r_k||^2, r_k the residual that entered the last
// iteration (rebuilt as r + alpha Ap).  Between replacements <r_{k+1}, r_k> vanishes up to
// rounding and this is ||r_{k+1}||^2 / ||r_k||^2; at a replacement the corrected residual
// is not the iterated one, and the Fletcher-Reeves form would carry a direction built with
// the rounded operator into it: with BF16 links on Haar links at m = 0.01 that form
// stalls near 1e-4, this one reaches 1e-10 (flexible CG: Golub & Ye 1999, Notay 2000).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <type_traits>
#include <vector>

#include "dslash_multi.cuh"
#include "dslash_paired.cuh"
#include "lqcd_internal.cuh"
#include "tma.cuh"
#include "tune.cuh"

bool dslash_vec_ok(lq_prec gauge, lq_prec vec);
lq_status launch_dslash_multi(lq_context* ctx, MultiKArgs a, lq_prec gp, int recon, lq_prec vp,
                              const std::string& key, cudaStream_t s);
lq_status launch_dslash_paired(lq_context* ctx, const lq_gauge* U, PairedKArgs k, int red_cols_max, int* cols_out,
                               cudaStream_t s);
PairedKArgs make_paired_kargs(const lq_gauge* U, const void* in, void* out, int out_parity, int nrhs);

namespace {

constexpr int kBlas = 256;  // threads per block of the vector kernels

template <class T> __device__ __forceinline__ double site_norm2(const T* v) {
  T s = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) s = fma(v[k], v[k], s);
  return (double)s;
}

// A vector of one rhs seen as 16-byte chunks (float4 for FP32, double2 for FP64): a
// site-ordered vector is contiguous and Vh * bytes_per_site is a multiple of 16 (Vh is
// a multiple of 8), so the BLAS kernels need no site structure and every access is a
// full-width, fully coalesced 16-byte load or store.
template <lq_prec VP> struct Chunk;
template <> struct Chunk<LQ_F32> {
  using real = float;
  using vec = float4;
  static constexpr int n = 4;
  __device__ __forceinline__ static void get(const vec& a, float* v) { v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; }
  __device__ __forceinline__ static vec put(const float* v) { return make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct Chunk<LQ_F64> {
  using real = double;
  using vec = double2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void get(const vec& a, double* v) { v[0] = a.x; v[1] = a.y; }
  __device__ __forceinline__ static vec put(const double* v) { return make_double2(v[0], v[1]); }
};

// alpha = rr / <p,Ap> for each rhs (one block per rhs): <p,Ap> arrives as the per-block
// partials of the preceding D_eo launch (FIN_DEFER, `cols` per rhs), summed here once in a
// fixed order.  A separate one-block launch: were every block of the update kernel to sum
// them, all of its blocks would hammer the same few L2 lines.
__global__ void __launch_bounds__(1024) k_cg_alpha(const double* pap, size_t stride, int cols, CGScalars* sc) {
  pdl_wait();
  const int rhs = blockIdx.x;
  const double pAp = block_total(pap + (size_t)rhs * stride, cols);
  if (threadIdx.x == 0) {
    CGScalars* s = sc + rhs;
    s->pAp = pAp;
    s->alpha = (s->active && pAp > 0.0) ? s->rr / pAp : 0.0;
    if (s->active) s->alpha_last = s->alpha;
  }
  pdl_trigger();
}

// <p,Ap> of the single-lattice solve in two stages, without a one-block launch: block g
// of a system sums columns g, g + kPapGroups, ... of the D_eo partials (FIN_DEFER) into
// gsum[rhs][g]; every block of k_cg_update then sums the kPapGroups values itself, in the
// same order (the same alpha in every block).  (k_cg_alpha, one 1024-thread block per
// system, spent ~7 us per iteration at 32^4 in its FP64 tree on one SM.)
constexpr int kPapGroups = 32;
__global__ void __launch_bounds__(256) k_cg_pap(const double* pap, size_t stride, int cols, double* gsum) {
  pdl_wait();
  const int rhs = blockIdx.y, g = blockIdx.x;
  const double* row = pap + (size_t)rhs * stride;
  double v[1] = {0.0};
  for (int b = g + kPapGroups * (int)threadIdx.x; b < cols; b += kPapGroups * (int)blockDim.x) v[0] += __ldcg(row + b);
  pdl_trigger();
  block_sum_store<1>(v, gsum + (size_t)rhs * kPapGroups + g, 1, 1);
}

// x += alpha p; r -= alpha Ap; ||r||^2 -> FIN_BETA.  grid = (nbx, nrhs), about two
// blocks per SM in all; each thread takes kUnroll chunks of its grid-stride sequence at a
// time (all their loads in flight together).  FP64 vectors: every square is accumulated
// in FP64.  FP32 vectors: each thread sums its squares in FP32 with Kahan compensation
// (error at most ~2 u of the sum, u = 2^-24: the rounding of one FP32 value), a warp sums
// its threads' values with the compensated FP32 tree (warp_sum), and the warps' sums are
// reduced in FP64.  On GB300's FP64 pipe (1/64 of FP32) an FP64
// conversion and add per real, or even per chunk, took as long as the memory traffic.
// (A TMA-tiled variant -- four bulk loads into shared memory, two bulk stores -- measured
// slower than the grid-stride form: 21.8 vs 20.1 us FP32, 44 vs 35 us FP64 at 32^4.)
constexpr int kUnroll = 4;
template <lq_prec VP>
__global__ void __launch_bounds__(kBlas, 2) k_cg_update(void* x, void* r, const void* p, const void* Ap,
                                                        const double* gsum, int Vh, Reducer red) {
  using C = Chunk<VP>;
  using T = typename C::real;
  using V = typename C::vec;
  const int rhs = blockIdx.y;
  const size_t nch = (size_t)Vh * VecT<VP>::bytes_per_site / 16;
  V* xc = reinterpret_cast<V*>(x) + rhs * nch;
  V* rc = reinterpret_cast<V*>(r) + rhs * nch;
  const V* pc = reinterpret_cast<const V*>(p) + rhs * nch;
  const V* ac = reinterpret_cast<const V*>(Ap) + rhs * nch;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  V xw[kUnroll], rw[kUnroll], pw[kUnroll], aw[kUnroll];
  auto load = [&](size_t b0) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const size_t i = b0 + u * stride;
      if (i < nch) {
        xw[u] = xc[i];
        rw[u] = rc[i];
        pw[u] = __ldg(pc + i);
        aw[u] = __ldg(ac + i);
      }
    }
  };
  pdl_wait();
  load(i0);   // the thread's first chunks are in flight while alpha is formed
  CGScalars* sc = reinterpret_cast<CGScalars*>(red.finisher_state) + rhs;
  // alpha = rr / <p,Ap> from the kPapGroups group sums (block 0 records it in the state;
  // the FIN_BETA finisher at the end reads none of these fields)
  __shared__ double s_alpha;
  if (threadIdx.x < 32) {
    double v = kPapGroups == 32 ? __ldcg(gsum + (size_t)rhs * kPapGroups + threadIdx.x) : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      const double a = (sc->active && v > 0.0) ? sc->rr / v : 0.0;
      s_alpha = a;
      if (blockIdx.x == 0) {
        sc->pAp = v;
        sc->alpha = a;
        if (sc->active) sc->alpha_last = a;
      }
    }
  }
  __syncthreads();
  const T alpha = (T)s_alpha;
  double acc[1] = {0.0};
  float ks = 0.f, kc = 0.f;   // FP32: compensated running sum (Kahan) and its correction
  for (; i0 < nch; i0 += kUnroll * stride) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const size_t i = i0 + u * stride;
      if (i >= nch) continue;
      T xv[C::n], rv[C::n], pv[C::n], av[C::n];
      C::get(xw[u], xv);
      C::get(rw[u], rv);
      C::get(pw[u], pv);
      C::get(aw[u], av);
#pragma unroll
      for (int k = 0; k < C::n; ++k) {
        xv[k] = fma(alpha, pv[k], xv[k]);
        rv[k] = fma(-alpha, av[k], rv[k]);
      }
      if constexpr (VP == LQ_F64) {
#pragma unroll
        for (int k = 0; k < C::n; ++k) acc[0] = fma((double)rv[k], (double)rv[k], acc[0]);
      } else {
#pragma unroll
        for (int k = 0; k < C::n; ++k) {
          const float y = fmaf(rv[k], rv[k], -kc);
          const float t = ks + y;
          kc = (t - ks) - y;
          ks = t;
        }
      }
      xc[i] = C::put(xv);
      rc[i] = C::put(rv);
    }
    if (i0 + kUnroll * stride < nch) load(i0 + kUnroll * stride);
  }
  pdl_trigger();
  if constexpr (VP == LQ_F64) {
    block_reduce<1>(acc, red, rhs, gridDim.y);
  } else {
    const float accf[1] = {ks - kc};   // the thread's sum, then the compensated warp tree
    block_reduce<1>(accf, red, rhs, gridDim.y);
  }
}

// The FP32 update of k_cg_update with its operands streamed through shared memory by TMA
// bulk copies: one block per SM, tiles of kUpdTile 16-byte chunks of x, r, p and Ap (64 KB)
// in a ring of kUpdStages stages.  Thread 0 issues the four copies of a tile kUpdStages - 1
// tiles ahead and waits for the current one on its mbarrier (bounded: on time-out it sets
// kDevTmaTimeout in *status, waits once more for every copy it issued and the block stops);
// the threads read the tile from shared memory and store x and r to global memory.  Two
// tiles (128 KB per SM) are always in flight, without registers holding them.
constexpr int kUpdTile = 1024;
constexpr int kUpdStages = 3;
constexpr size_t kUpdSmem = (size_t)kUpdStages * 4 * kUpdTile * sizeof(float4);
__global__ void __launch_bounds__(kBlas, 1) k_cg_update_tma(float4* x, float4* r, const float4* p, const float4* Ap,
                                                            const double* gsum, int Vh, Reducer red,
                                                            unsigned int* status) {
  extern __shared__ __align__(128) unsigned char upd_raw[];
  float4* stg = reinterpret_cast<float4*>(upd_raw);   // [stage][x, r, p, Ap][kUpdTile]
  __shared__ uint64_t bar[kUpdStages];
  __shared__ int ok_s;
  __shared__ double s_alpha;
  const int rhs = blockIdx.y;
  const size_t nch = (size_t)Vh * 3 / 2;              // 24 bytes per site, 16 per chunk
  float4* xc = x + rhs * nch;
  float4* rc = r + rhs * nch;
  const float4* pc = p + rhs * nch;
  const float4* ac = Ap + rhs * nch;
  const size_t ntile = (nch + kUpdTile - 1) / kUpdTile;
  const int nmine = blockIdx.x < ntile ? (int)((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kUpdStages; ++k) tma::mbar_init(&bar[k], 1);
  }
  __syncthreads();
  pdl_wait();
  auto tile_of = [&](int k, size_t& c0, uint32_t& n) {
    c0 = ((size_t)blockIdx.x + (size_t)k * gridDim.x) * kUpdTile;
    n = (uint32_t)(nch - c0 < (size_t)kUpdTile ? nch - c0 : (size_t)kUpdTile);
  };
  auto issue = [&](int k) {   // thread 0: tile k of this block into stage k % kUpdStages
    size_t c0;
    uint32_t n;
    tile_of(k, c0, n);
    uint64_t* b = &bar[k % kUpdStages];
    float4* sg = stg + (size_t)(k % kUpdStages) * 4 * kUpdTile;
    tma::mbar_expect_tx(b, 4 * n * (uint32_t)sizeof(float4));
    tma::load(sg, xc + c0, n * sizeof(float4), b);
    tma::load(sg + kUpdTile, rc + c0, n * sizeof(float4), b);
    tma::load(sg + 2 * kUpdTile, pc + c0, n * sizeof(float4), b);
    tma::load(sg + 3 * kUpdTile, ac + c0, n * sizeof(float4), b);
  };
  int issued = 0;
  if (threadIdx.x == 0)
    for (; issued < kUpdStages - 1 && issued < nmine; ++issued) issue(issued);
  CGScalars* sc = reinterpret_cast<CGScalars*>(red.finisher_state) + rhs;
  if (threadIdx.x < 32) {   // alpha = rr / <p,Ap> from the kPapGroups group sums
    double v = __ldcg(gsum + (size_t)rhs * kPapGroups + threadIdx.x);
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      const double a = (sc->active && v > 0.0) ? sc->rr / v : 0.0;
      s_alpha = a;
      if (blockIdx.x == 0) {
        sc->pAp = v;
        sc->alpha = a;
        if (sc->active) sc->alpha_last = a;
      }
    }
  }
  __syncthreads();
  const float alpha = (float)s_alpha;
  float ks = 0.f, kc = 0.f;
  for (int k = 0; k < nmine; ++k) {
    if (threadIdx.x == 0) {
      if (issued < nmine) issue(issued++);   // into the stage freed at the end of tile k - 1
      int ok = tma::mbar_wait(&bar[k % kUpdStages], (k / kUpdStages) & 1) ? 1 : 0;
      if (!ok) {
        atomicOr(status, kDevTmaTimeout);
        for (int j = k; j < issued; ++j) tma::mbar_wait(&bar[j % kUpdStages], (j / kUpdStages) & 1);
      }
      ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) break;   // copies that did not arrive: the block stops (the solve reports it)
    size_t c0;
    uint32_t n;
    tile_of(k, c0, n);
    const float4* sg = stg + (size_t)(k % kUpdStages) * 4 * kUpdTile;
#pragma unroll
    for (int j = 0; j < kUpdTile / kBlas; ++j) {
      const uint32_t i = threadIdx.x + j * kBlas;
      if (i >= n) break;
      float4 xv = sg[i], rv = sg[kUpdTile + i];
      const float4 pv = sg[2 * kUpdTile + i], av = sg[3 * kUpdTile + i];
      xv.x = fmaf(alpha, pv.x, xv.x); xv.y = fmaf(alpha, pv.y, xv.y);
      xv.z = fmaf(alpha, pv.z, xv.z); xv.w = fmaf(alpha, pv.w, xv.w);
      rv.x = fmaf(-alpha, av.x, rv.x); rv.y = fmaf(-alpha, av.y, rv.y);
      rv.z = fmaf(-alpha, av.z, rv.z); rv.w = fmaf(-alpha, av.w, rv.w);
      const float q[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float y = fmaf(q[m], q[m], -kc);
        const float t = ks + y;
        kc = (t - ks) - y;
        ks = t;
      }
      xc[c0 + i] = xv;
      rc[c0 + i] = rv;
    }
    __syncthreads();   // stage k % kUpdStages is free again
  }
  pdl_trigger();
  const float accf[1] = {ks - kc};
  block_reduce<1>(accf, red, rhs, gridDim.y);
}

// p = r + beta p for active right-hand sides.  grid = (nbx, nrhs), about one wave of
// blocks (four per SM) in all, 16-byte chunks, kUnroll chunks of the thread's grid-stride
// sequence loaded together.
template <lq_prec VP>
__global__ void __launch_bounds__(kBlas, 4) k_cg_xpay(const void* r, void* p, const CGScalars* sc, int Vh) {
  using C = Chunk<VP>;
  using T = typename C::real;
  using V = typename C::vec;
  const int rhs = blockIdx.y;
  const size_t nch = (size_t)Vh * VecT<VP>::bytes_per_site / 16;
  const V* rc = reinterpret_cast<const V*>(r) + rhs * nch;
  V* pc = reinterpret_cast<V*>(p) + rhs * nch;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  constexpr int kU = VP == LQ_F64 ? 2 : kUnroll;   // (FP64: four would spill)
  size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  V rw[kU], pw[kU];
  auto load = [&](size_t b0) {
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * stride;
      if (i < nch) {
        rw[u] = __ldg(rc + i);
        pw[u] = pc[i];
      }
    }
  };
  pdl_wait();
  load(i0);   // in flight while the scalars are read (wasted only for an inactive rhs)
  if (sc[rhs].active) {
    const T beta = (T)sc[rhs].beta;
    for (; i0 < nch; i0 += kU * stride) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const size_t i = i0 + u * stride;
        if (i >= nch) continue;
        T rv[C::n], pv[C::n];
        C::get(rw[u], rv);
        C::get(pw[u], pv);
#pragma unroll
        for (int k = 0; k < C::n; ++k) pv[k] = fma(beta, pv[k], rv[k]);
        pc[i] = C::put(pv);
      }
      if (i0 + kU * stride < nch) load(i0 + kU * stride);
    }
  }
  pdl_trigger();
}

// dst (precision VD) = src (precision VS) for every rhs; optional ||dst||^2 -> FIN_STORE.
template <lq_prec VS, lq_prec VD>
__global__ void __launch_bounds__(kBlas) k_convert(const void* src, void* dst, int Vh, int reduce, Reducer red) {
  using S = VecT<VS>;
  using D = VecT<VD>;
  const int rhs = blockIdx.y;
  pdl_wait();
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

// Residual replacement: r = round(r_hi) for every rhs, with two FP64 sums per rhs into
// the FIN_STORE rows 2 rhs and 2 rhs + 1: ||r_new||^2 and, when `with_dot`,
// Re<r_new, r_k> with r_k = r_old + alpha_last Ap rebuilt from the iterated residual r_old
// this launch overwrites (the Polak-Ribiere beta of the replacement).
template <lq_prec VL>
__global__ void __launch_bounds__(kBlas) k_cg_replace(const double* rhi, void* r, const void* Ap, const CGScalars* sc,
                                                      int Vh, int with_dot, Reducer red) {
  using L = VecT<VL>;
  using T = typename L::real;
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * Vh;
  const T alpha = with_dot ? (T)sc[rhs].alpha_last : T(0);
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    double h[6];
    T n[6];
    VecT<LQ_F64>::load(rhi, off + i, h);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      n[k] = (T)h[k];
      acc[0] = fma((double)n[k], (double)n[k], acc[0]);
    }
    if (with_dot) {
      T o[6], a[6];
      L::load_rw(r, off + i, o);
      L::load(Ap, off + i, a);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[1] = fma((double)n[k], (double)fma(alpha, a[k], o[k]), acc[1]);
    }
    L::store(r, off + i, n);
  }
  block_reduce<2>(acc, red, 2 * rhs, 2 * gridDim.y, blockIdx.x, gridDim.x);
}

// x_hi += x_lo; x_lo = 0.
template <lq_prec VL>
__global__ void __launch_bounds__(kBlas) k_fold(double* x_hi, void* x_lo, int Vh) {
  using L = VecT<VL>;
  const int rhs = blockIdx.y;
  pdl_wait();
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


// ------------------------------------------------- paired-layout (multi-RHS) kernels ---
//
// The multi-RHS mixed solve keeps its FP32 inner vectors in the paired colour-planar
// layout of dslash_eo_paired: pair pr = (rhs 2 pr, 2 pr + 1) is 3 Vh float4 chunks
// (Re a, Re b, Im a, Im b); lanes x, z belong to rhs a, y, w to rhs b.  A padding half (odd
// nrhs) is never active: its scalars are not read, its partials not stored.

// p = r + beta p for the active right-hand sides of each pair.  grid = (nbx, npair).
__global__ void __launch_bounds__(kBlas, 4) k_cgp_xpay(const float4* r, float4* p, const CGScalars* sc, int Vh,
                                                       int nrhs) {
  const int pr = blockIdx.y, ra = 2 * pr, rb = 2 * pr + 1;
  const size_t nch = (size_t)3 * Vh;
  const float4* rc = r + pr * nch;
  float4* pc = p + pr * nch;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float4 rw[kUnroll], pw[kUnroll];
  auto load = [&](size_t b0) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const size_t i = b0 + u * stride;
      if (i < nch) {
        rw[u] = __ldg(rc + i);
        pw[u] = pc[i];
      }
    }
  };
  pdl_wait();
  load(i0);   // in flight while the scalars are read
  const bool actA = sc[ra].active != 0, actB = rb < nrhs && sc[rb].active != 0;
  if (actA || actB) {
    const float bA = actA ? (float)sc[ra].beta : 0.f, bB = actB ? (float)sc[rb].beta : 0.f;
    for (; i0 < nch; i0 += kUnroll * stride) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const size_t i = i0 + u * stride;
        if (i >= nch) continue;
        float4 q = pw[u];
        if (actA) {
          q.x = fmaf(bA, q.x, rw[u].x);
          q.z = fmaf(bA, q.z, rw[u].z);
        }
        if (actB) {
          q.y = fmaf(bB, q.y, rw[u].y);
          q.w = fmaf(bB, q.w, rw[u].w);
        }
        pc[i] = q;
      }
      if (i0 + kUnroll * stride < nch) load(i0 + kUnroll * stride);
    }
  }
  pdl_trigger();
}

// x += alpha p; r -= alpha Ap; ||r||^2 -> FIN_BETA, per rhs of each pair, alpha of each
// rhs from its kPapGroups group sums of <p,Ap> (as k_cg_update).  grid = (nbx, npair).
__global__ void __launch_bounds__(kBlas, 2) k_cgp_update(float4* x, float4* r, const float4* p, const float4* Ap,
                                                         const double* gsum, int Vh, int nrhs, Reducer red) {
  const int pr = blockIdx.y;
  const size_t nch = (size_t)3 * Vh;
  float4* xc = x + pr * nch;
  float4* rc = r + pr * nch;
  const float4* pc = p + pr * nch;
  const float4* ac = Ap + pr * nch;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float4 xw[kUnroll], rw[kUnroll], pw[kUnroll], aw[kUnroll];
  auto load = [&](size_t b0) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const size_t i = b0 + u * stride;
      if (i < nch) {
        xw[u] = xc[i];
        rw[u] = rc[i];
        pw[u] = __ldg(pc + i);
        aw[u] = __ldg(ac + i);
      }
    }
  };
  pdl_wait();
  load(i0);   // in flight while alpha is formed
  CGScalars* sc = reinterpret_cast<CGScalars*>(red.finisher_state);
  __shared__ double s_alpha[2];
  if (threadIdx.x < 64) {   // warp 0: rhs 2 pr, warp 1: rhs 2 pr + 1
    const int h = threadIdx.x >> 5, rh = 2 * pr + h;
    double v = rh < nrhs ? __ldcg(gsum + (size_t)rh * kPapGroups + (threadIdx.x & 31)) : 0.0;
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) {
      double a = 0.0;
      if (rh < nrhs) {
        CGScalars* c = sc + rh;
        a = (c->active && v > 0.0) ? c->rr / v : 0.0;
        if (blockIdx.x == 0) {
          c->pAp = v;
          c->alpha = a;
          if (c->active) c->alpha_last = a;
        }
      }
      s_alpha[h] = a;
    }
  }
  __syncthreads();
  const float aA = (float)s_alpha[0], aB = (float)s_alpha[1];
  float sA = 0.f, cA = 0.f, sB = 0.f, cB = 0.f;   // Kahan sums of each rhs's squares
  auto kahan = [](float& s_, float& c_, float v) {
    const float y = v - c_;
    const float t = s_ + y;
    c_ = (t - s_) - y;
    s_ = t;
  };
  for (; i0 < nch; i0 += kUnroll * stride) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const size_t i = i0 + u * stride;
      if (i >= nch) continue;
      float4 xv = xw[u], rv = rw[u];
      xv.x = fmaf(aA, pw[u].x, xv.x); xv.z = fmaf(aA, pw[u].z, xv.z);
      xv.y = fmaf(aB, pw[u].y, xv.y); xv.w = fmaf(aB, pw[u].w, xv.w);
      rv.x = fmaf(-aA, aw[u].x, rv.x); rv.z = fmaf(-aA, aw[u].z, rv.z);
      rv.y = fmaf(-aB, aw[u].y, rv.y); rv.w = fmaf(-aB, aw[u].w, rv.w);
      kahan(sA, cA, fmaf(rv.x, rv.x, rv.z * rv.z));
      kahan(sB, cB, fmaf(rv.y, rv.y, rv.w * rv.w));
      xc[i] = xv;
      rc[i] = rv;
    }
    if (i0 + kUnroll * stride < nch) load(i0 + kUnroll * stride);
  }
  pdl_trigger();
  const float acc[2] = {sA - cA, sB - cB};
  block_reduce<2>(acc, red, 2 * pr, nrhs, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------- segmented (multi-lattice) kernels -
//
// The batched solver keeps every vector of all its lattices in one concatenated array:
// lattice l starts at site voff_l and holds [nrhs][Vh_l][3].  A "segment" is one
// (lattice, rhs) system, q = l * nrhs + rhs.  The kernels below walk tiles of kBlas sites
// of the segments with a persistent grid; per-segment reductions go through per-tile
// partials and the last block (grid_finish).

struct SegLat {
  size_t voff;   // first site of the lattice
  int Vh;        // sites per rhs
  int tile0;     // first tile of the lattice
  int tps;       // tiles per segment
};

struct SegArgs {
  int nlat, nrhs, ntiles;
  size_t pstride;
  SegLat lat[kMaxLat];
};

__device__ __forceinline__ void seg_locate(const SegArgs& g, int tile, int& q, size_t& base, int& chunk, int& Vh,
                                           int& l) {
  l = 0;
  while (l + 1 < g.nlat && tile >= g.lat[l + 1].tile0) ++l;
  const int t = tile - g.lat[l].tile0;
  const int rhs = t / g.lat[l].tps;
  chunk = t % g.lat[l].tps;
  q = l * g.nrhs + rhs;
  Vh = g.lat[l].Vh;
  base = g.lat[l].voff + (size_t)rhs * Vh;
}

template <lq_prec VP>
__global__ void __launch_bounds__(kBlas) k_seg_update(void* x, void* r, const void* p, const void* Ap,
                                                      const SegArgs g, Reducer red) {
  using VT = VecT<VP>;
  using T = typename VT::real;
  const CGScalars* sc = reinterpret_cast<const CGScalars*>(red.finisher_state);
  using A = typename std::conditional<VP == LQ_F64, double, float>::type;
  for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    int q, chunk, Vh, l;
    size_t base;
    seg_locate(g, tile, q, base, chunk, Vh, l);
    // FP32 vectors: the site's squares in FP32, the tile's sum by the compensated FP32
    // block tree (block_sum_f32) and FP64 above
    A acc[1] = {A(0)};
    const int i = chunk * kBlas + threadIdx.x;
    if (sc[q].active && i < Vh) {
      const T alpha = (T)sc[q].alpha;
      T xv[6], rv[6], pv[6], av[6];
      VT::load_rw(x, base + i, xv);
      VT::load_rw(r, base + i, rv);
      VT::load(p, base + i, pv);
      VT::load(Ap, base + i, av);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        xv[k] = fma(alpha, pv[k], xv[k]);
        rv[k] = fma(-alpha, av[k], rv[k]);
      }
      VT::store(x, base + i, xv);
      VT::store(r, base + i, rv);
      if constexpr (VP == LQ_F64) {
        acc[0] = site_norm2(rv);
      } else {
        float s2 = rv[0] * rv[0];
#pragma unroll
        for (int k = 1; k < 6; ++k) s2 = fmaf(rv[k], rv[k], s2);
        acc[0] = s2;
      }
    }
    block_sum_store<1>(acc, red.partials + (size_t)q * g.pstride + chunk, g.pstride, 1);
  }
  grid_finish(red, g.nlat * g.nrhs, g.pstride, [&](int q) { return g.lat[q / g.nrhs].tps; });
}

template <lq_prec VP>
__global__ void __launch_bounds__(kBlas) k_seg_xpay(const void* r, void* p, const CGScalars* sc, const SegArgs g) {
  using VT = VecT<VP>;
  using T = typename VT::real;
  for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    int q, chunk, Vh, l;
    size_t base;
    seg_locate(g, tile, q, base, chunk, Vh, l);
    const int i = chunk * kBlas + threadIdx.x;
    if (!sc[q].active || i >= Vh) continue;
    const T beta = (T)sc[q].beta;
    T rv[6], pv[6];
    VT::load(r, base + i, rv);
    VT::load_rw(p, base + i, pv);
#pragma unroll
    for (int k = 0; k < 6; ++k) pv[k] = fma(beta, pv[k], rv[k]);
    VT::store(p, base + i, pv);
  }
}

// dst = src for every system (mask NULL) or for the systems with mask[q].ru set; ||dst||^2
// of those systems -> FIN_STORE (0 for the others).
template <lq_prec VS, lq_prec VD>
__global__ void __launch_bounds__(kBlas) k_seg_convert(const void* src, void* dst, const SegArgs g, Reducer red,
                                                       const CGScalars* mask) {
  using Sv = VecT<VS>;
  using Dv = VecT<VD>;
  for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    int q, chunk, Vh, l;
    size_t base;
    seg_locate(g, tile, q, base, chunk, Vh, l);
    const int i = chunk * kBlas + threadIdx.x;
    double acc[1] = {0.0};
    if (i < Vh && (!mask || mask[q].ru)) {
      typename Sv::real a[6];
      typename Dv::real b[6];
      Sv::load(src, base + i, a);
#pragma unroll
      for (int k = 0; k < 6; ++k) b[k] = (typename Dv::real)a[k];
      Dv::store(dst, base + i, b);
      double s2 = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s2 += (double)b[k] * (double)b[k];
      acc[0] = s2;
    }
    block_sum_store<1>(acc, red.partials + (size_t)q * g.pstride + chunk, g.pstride, 1);
  }
  grid_finish(red, g.nlat * g.nrhs, g.pstride, [&](int q) { return g.lat[q / g.nrhs].tps; });
}

// Batched residual replacement of the systems whose ru flag is set: r = round(r_hi), with
// ||r_new||^2 and Re<r_new, r_old + alpha_last Ap> into FIN_STORE rows 2q and 2q + 1
// (zeros for the other systems); see k_cg_replace.
template <lq_prec VL>
__global__ void __launch_bounds__(kBlas) k_seg_replace(const double* rhi, void* r, const void* Ap, const SegArgs g,
                                                       Reducer red, const CGScalars* sc) {
  using L = VecT<VL>;
  using T = typename L::real;
  for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    int q, chunk, Vh, l;
    size_t base;
    seg_locate(g, tile, q, base, chunk, Vh, l);
    const int i = chunk * kBlas + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (i < Vh && sc[q].ru) {
      const T alpha = (T)sc[q].alpha_last;
      double h[6];
      T n[6], o[6], a[6];
      VecT<LQ_F64>::load(rhi, base + i, h);
      L::load_rw(r, base + i, o);
      L::load(Ap, base + i, a);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        n[k] = (T)h[k];
        acc[0] = fma((double)n[k], (double)n[k], acc[0]);
        acc[1] = fma((double)n[k], (double)fma(alpha, a[k], o[k]), acc[1]);
      }
      L::store(r, base + i, n);
    }
    block_sum_store<2>(acc, red.partials + (size_t)(2 * q) * g.pstride + chunk, g.pstride, 2);
  }
  grid_finish(red, 2 * g.nlat * g.nrhs, g.pstride, [&](int q2) { return g.lat[(q2 / 2) / g.nrhs].tps; });
}

template <lq_prec VL>
__global__ void __launch_bounds__(kBlas) k_seg_fold(double* x_hi, void* x_lo, const SegArgs g) {
  using L = VecT<VL>;
  for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    int q, chunk, Vh, l;
    size_t base;
    seg_locate(g, tile, q, base, chunk, Vh, l);
    const int i = chunk * kBlas + threadIdx.x;
    if (i >= Vh) continue;
    typename L::real a[6], z[6];
    double h[6];
    L::load_rw(x_lo, base + i, a);
    VecT<LQ_F64>::load_rw(x_hi, base + i, h);
#pragma unroll
    for (int k = 0; k < 6; ++k) { h[k] += (double)a[k]; z[k] = 0; }
    VecT<LQ_F64>::store(x_hi, base + i, h);
    L::store(x_lo, base + i, z);
  }
}

// Lattice set of a batched solve.
struct Batch {
  int nlat;
  const lq_gauge* hi[kMaxLat];
  const lq_gauge* lo[kMaxLat];   // == hi for the plain FP64 solve
  double mass[kMaxLat];
  size_t voff[kMaxLat];
  SegArgs seg;
  int seg_grid;
  std::string key_lo, key_hi;     // tuning keys of the two multi-lattice Dslash formats
};

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
  bool paired = false;   // FP32 inner vectors in the paired colour-planar layout (nrhs >= 2)
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
  double* dpartials;     // [nrhs][nblocks_max]: <p,Ap> partials of D_eo (k_cg_pap / k_cg_alpha)
  double* gsum;          // [nrhs][kPapGroups]: <p,Ap> group sums (k_cg_pap -> k_cg_update)
  unsigned int* counter;
  int nblocks_max;
  bool pdl = false;      // programmatic dependent launch for the iteration kernels
  int nsys = 0;          // independent systems: nrhs, or nlat * nrhs when batched
  size_t sites = 0;      // sites of one full vector (all systems)
  const Batch* batch = nullptr;

  Reducer reducer(int fin) const {
    return Reducer{partials, counter, result, nblocks_max, fin, (void*)sc};
  }
  size_t vbytes(lq_prec q) const { return sites * 6 * lq_prec_bytes(q); }
  // bytes of one inner vector: canonical, or paired (an odd nrhs pads its last pair)
  size_t vin_bytes() const { return paired ? (size_t)((nrhs + 1) / 2) * 3 * Vh * 16 : vbytes(vp); }
};

// ---- batched (multi-lattice) versions of the solver steps

// Multi-lattice launch arguments over the concatenated vectors (lattice l at site offset
// voff_l); w1, w2 may be NULL.
MultiKArgs multi_args(const Solver& S, bool hi, int out_par, const void* in, void* out, const void* w1 = nullptr,
                      const void* w2 = nullptr) {
  const Batch& B = *S.batch;
  const size_t bps = hi || !S.mixed ? 48 : 24;  // bytes per site of the vectors
  MultiKArgs a;
  memset(&a, 0, sizeof a);
  a.nlat = B.nlat;
  a.nrhs = S.nrhs;
  a.out_par = out_par;
  a.c = 1.0;
  a.reduce = RED_NONE;
  a.pstride = (size_t)S.nblocks_max;
  for (int l = 0; l < B.nlat; ++l) {
    const lq_gauge* g = hi ? B.hi[l] : B.lo[l];
    const size_t off = B.voff[l] * bps;
    a.lat[l].gauge = g->data;
    a.lat[l].blk_bytes = g->blk_bytes;
    a.lat[l].G = make_geom(g);
    a.lat[l].in = (const char*)in + off;
    a.lat[l].out = (char*)out + off;
    a.lat[l].w1 = w1 ? (const char*)w1 + off : nullptr;
    a.lat[l].w2 = w2 ? (const char*)w2 + off : nullptr;
  }
  return a;
}

lq_status batch_iteration_dslash(Solver& S) {
  const Batch& B = *S.batch;
  const lq_gauge* g0 = B.lo[0];
  MultiKArgs d = multi_args(S, false, 1, S.p, S.t);
  lq_status st = launch_dslash_multi(S.ctx, d, g0->prec, g0->recon, S.vp, B.key_lo, S.s);
  if (st) return st;
  // Ap = m^2 p - D_eo t with <p, Ap>: per-block row partials only (FIN_DEFER), summed by
  // k_cg_alpha with one block per system (a last-block finisher would sum every row alone)
  MultiKArgs e = multi_args(S, false, 0, S.t, S.Ap, S.p);
  for (int l = 0; l < B.nlat; ++l) e.lat[l].a1 = B.mass[l] * B.mass[l];
  e.c = -1.0;
  e.reduce = RED_DOT;
  e.red = S.reducer(FIN_DEFER);
  e.red.partials = S.dpartials;
  e.skip_state = S.sc;
  e.skip_mode = SKIP_INACTIVE;
  int cols = 0;
  e.cols_out = &cols;
  st = launch_dslash_multi(S.ctx, e, g0->prec, g0->recon, S.vp, B.key_lo, S.s);
  if (st) return st;
  if (cols < 1) return lq_fail(S.ctx, LQ_ERR_INVALID_ARG, "internal: empty reduction launch");
  k_cg_alpha<<<S.nsys, 1024, 0, S.s>>>(S.dpartials, e.pstride, cols, S.sc);
  LQ_CHECK_LAUNCH(S.ctx, "k_cg_alpha");
  return LQ_OK;
}

// skip_done: leave out the lattices whose systems have all met the tolerance already
// (their residual and norm entries are then not rewritten).
lq_status batch_true_residual(Solver& S, int skip_mode) {
  const Batch& B = *S.batch;
  const lq_gauge* g0 = B.hi[0];
  MultiKArgs d = multi_args(S, true, 1, S.x, S.thi);
  if (skip_mode) {
    d.skip_state = S.sc;
    d.skip_mode = skip_mode;
  }
  lq_status st = launch_dslash_multi(S.ctx, d, g0->prec, g0->recon, LQ_F64, B.key_hi, S.s);
  if (st) return st;
  MultiKArgs e = multi_args(S, true, 0, S.thi, S.rhi, S.b, S.x);
  if (skip_mode) {
    e.skip_state = S.sc;
    e.skip_mode = skip_mode;
  }
  for (int l = 0; l < B.nlat; ++l) {
    e.lat[l].a1 = 1.0;
    e.lat[l].a2 = -B.mass[l] * B.mass[l];
  }
  e.c = 1.0;
  e.reduce = RED_NORM;
  e.red = S.reducer(FIN_STORE);
  return launch_dslash_multi(S.ctx, e, g0->prec, g0->recon, LQ_F64, B.key_hi, S.s);
}

lq_status launch_blas_update(Solver& S) {
  if (S.batch) {
    const Batch& B = *S.batch;
    Reducer red = S.reducer(FIN_BETA);
    if (S.vp == LQ_F64) k_seg_update<LQ_F64><<<B.seg_grid, kBlas, 0, S.s>>>(S.xl, S.r, S.p, S.Ap, B.seg, red);
    else k_seg_update<LQ_F32><<<B.seg_grid, kBlas, 0, S.s>>>(S.xl, S.r, S.p, S.Ap, B.seg, red);
    LQ_CHECK_LAUNCH(S.ctx, "k_seg_update");
    return LQ_OK;
  }
  // about two blocks per SM over all right-hand sides: fewer block reductions (FP64), each
  // thread streaming more chunks
  Reducer red = S.reducer(FIN_BETA);
  if (S.vp == LQ_F32 && S.nrhs == 1) {
    // one block per SM, operands through shared memory by TMA.  Measured at 32^4: 104.2
    // against 105.2 us per FP32-12 iteration; with 8 right-hand sides (19 blocks each) the
    // register-staged kernel below is faster (162.9 against 164.4 us at 24^4).
    LQ_CUDA(S.ctx, cudaFuncSetAttribute(k_cg_update_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kUpdSmem));
    const int nt = std::max(1, (S.ctx->num_sms + S.nrhs - 1) / S.nrhs);
    cudaError_t e = launch_k(k_cg_update_tma, dim3(nt, S.nrhs), dim3(kBlas), kUpdSmem, S.s, S.pdl, (float4*)S.xl,
                             (float4*)S.r, (const float4*)S.p, (const float4*)S.Ap, (const double*)S.gsum, S.Vh, red,
                             S.ctx->dev_status);
    if (e != cudaSuccess) return lq_cuda_fail(S.ctx, e, "k_cg_update_tma");
    return LQ_OK;
  }
  const int nb = std::min(S.nbx, std::max(1, (2 * S.ctx->num_sms + S.nrhs - 1) / S.nrhs));
  dim3 grid(nb, S.nrhs);
  cudaError_t e = S.vp == LQ_F64
                      ? launch_k(k_cg_update<LQ_F64>, grid, dim3(kBlas), 0, S.s, S.pdl, S.xl, S.r, (const void*)S.p,
                                 (const void*)S.Ap, (const double*)S.gsum, S.Vh, red)
                      : launch_k(k_cg_update<LQ_F32>, grid, dim3(kBlas), 0, S.s, S.pdl, S.xl, S.r, (const void*)S.p,
                                 (const void*)S.Ap, (const double*)S.gsum, S.Vh, red);
  if (e != cudaSuccess) return lq_cuda_fail(S.ctx, e, "k_cg_update");
  return LQ_OK;
}

lq_status launch_xpay(Solver& S) {
  if (S.batch) {
    const Batch& B = *S.batch;
    if (S.vp == LQ_F64) k_seg_xpay<LQ_F64><<<B.seg_grid, kBlas, 0, S.s>>>(S.r, S.p, S.sc, B.seg);
    else k_seg_xpay<LQ_F32><<<B.seg_grid, kBlas, 0, S.s>>>(S.r, S.p, S.sc, B.seg);
    LQ_CHECK_LAUNCH(S.ctx, "k_seg_xpay");
    return LQ_OK;
  }
  const int nb = std::min(S.nbx, std::max(1, (4 * S.ctx->num_sms + S.nrhs - 1) / S.nrhs));
  dim3 grid(nb, S.nrhs);
  cudaError_t e = S.vp == LQ_F64
                      ? launch_k(k_cg_xpay<LQ_F64>, grid, dim3(kBlas), 0, S.s, S.pdl, (const void*)S.r, S.p,
                                 (const CGScalars*)S.sc, S.Vh)
                      : launch_k(k_cg_xpay<LQ_F32>, grid, dim3(kBlas), 0, S.s, S.pdl, (const void*)S.r, S.p,
                                 (const CGScalars*)S.sc, S.Vh);
  if (e != cudaSuccess) return lq_cuda_fail(S.ctx, e, "k_cg_xpay");
  return LQ_OK;
}

// One inner iteration.
// One inner iteration on the paired layout: xpay, D_oe and D_eo with <p,Ap> in the paired
// kernel, the group sums, the update.
lq_status iteration_paired(Solver& S) {
  const int npair = (S.nrhs + 1) / 2;
  {
    const int nb = std::min(S.nbx, std::max(1, (4 * S.ctx->num_sms + npair - 1) / npair));
    cudaError_t e = launch_k(k_cgp_xpay, dim3(nb, npair), dim3(kBlas), 0, S.s, S.pdl, (const float4*)S.r,
                             (float4*)S.p, (const CGScalars*)S.sc, S.Vh, S.nrhs);
    if (e != cudaSuccess) return lq_cuda_fail(S.ctx, e, "k_cgp_xpay");
  }
  PairedKArgs d = make_paired_kargs(S.Ulo, S.p, S.t, 1, S.nrhs);
  d.pdl = S.pdl ? 1 : 0;
  lq_status st = launch_dslash_paired(S.ctx, S.Ulo, d, 0, nullptr, S.s);
  if (st) return st;
  PairedKArgs e = make_paired_kargs(S.Ulo, S.t, S.Ap, 0, S.nrhs);
  e.pdl = S.pdl ? 1 : 0;
  e.w1 = (const float4*)S.p;
  e.a1 = (float)(S.mass * S.mass);
  e.c = -1.f;
  e.reduce = RED_DOT;
  e.red = S.reducer(FIN_DEFER);
  e.red.partials = S.dpartials;
  int cols = 0;
  st = launch_dslash_paired(S.ctx, S.Ulo, e, S.nblocks_max, &cols, S.s);
  if (st) return st;
  cudaError_t ce = launch_k(k_cg_pap, dim3(kPapGroups, S.nrhs), dim3(256), 0, S.s, S.pdl, (const double*)S.dpartials,
                            (size_t)cols, cols, S.gsum);
  if (ce != cudaSuccess) return lq_cuda_fail(S.ctx, ce, "k_cg_pap");
  const int nb = std::min(S.nbx, std::max(1, (2 * S.ctx->num_sms + npair - 1) / npair));
  ce = launch_k(k_cgp_update, dim3(nb, npair), dim3(kBlas), 0, S.s, S.pdl, (float4*)S.xl, (float4*)S.r,
                (const float4*)S.p, (const float4*)S.Ap, (const double*)S.gsum, S.Vh, S.nrhs,
                S.reducer(FIN_BETA));
  if (ce != cudaSuccess) return lq_cuda_fail(S.ctx, ce, "k_cgp_update");
  return LQ_OK;
}

lq_status iteration(Solver& S) {
  if (S.paired) return iteration_paired(S);
  lq_status st = launch_xpay(S);
  if (st) return st;
  if (S.batch) {
    st = batch_iteration_dslash(S);
    if (st) return st;
    return launch_blas_update(S);
  }
  DslashArgs d;
  d.U = S.Ulo;
  d.in = S.p;
  d.out = S.t;
  d.out_parity = 1;
  d.nrhs = S.nrhs;
  d.vec_prec = S.vp;
  d.rhs_stride = S.Vh;
  d.pdl = S.pdl;
  st = launch_dslash(S.ctx, d, S.s);
  if (st) return st;
  Reducer red = S.reducer(FIN_DEFER);
  red.partials = S.dpartials;
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
  cudaError_t ce = launch_k(k_cg_pap, dim3(kPapGroups, S.nrhs), dim3(256), 0, S.s, S.pdl, (const double*)S.dpartials,
                            (size_t)red.cols, red.cols, S.gsum);
  if (ce != cudaSuccess) return lq_cuda_fail(S.ctx, ce, "k_cg_pap");
  return launch_blas_update(S);
}

// r_hi = b - M x_hi in FP64 and ||r_hi||^2 -> result (FIN_STORE).
// r_hi = b - M x_hi in FP64 with ||r_hi||^2 -> result.  Batched, `skip_mode` (SKIP_DONE,
// SKIP_NO_RU) leaves out the lattice tiles whose systems are all skipped.
lq_status true_residual(Solver& S, int skip_mode = 0) {
  if (S.batch) return batch_true_residual(S, skip_mode);
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
  if (S.batch) {
    k_seg_fold<LQ_F32><<<S.batch->seg_grid, kBlas, 0, S.s>>>(S.x, S.xl, S.batch->seg);
    LQ_CHECK_LAUNCH(S.ctx, "k_seg_fold");
    return LQ_OK;
  }
  dim3 grid(S.nbx, S.nrhs);
  if (S.paired) {
    // x_lo to the canonical layout in t, folded from there; x_lo = 0
    lq_status st = lq_vec_unpair(S.ctx, S.Vh, S.nrhs, S.xl, S.t, S.s);
    if (st) return st;
    k_fold<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.x, S.t, S.Vh);
    LQ_CHECK_LAUNCH(S.ctx, "k_fold");
    LQ_CUDA(S.ctx, cudaMemsetAsync(S.xl, 0, S.vin_bytes(), S.s));
    return LQ_OK;
  }
  k_fold<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.x, S.xl, S.Vh);
  LQ_CHECK_LAUNCH(S.ctx, "k_fold");
  return LQ_OK;
}

// r_lo = round(r_hi) with ||r_lo||^2 -> result[2 i] and, when `with_dot` (a replacement
// during the iteration), Re<r_lo, r_k> -> result[2 i + 1] for the Polak-Ribiere beta.
// Batched: only the systems whose ru flag is set (always with the dot).
lq_status replace_residual(Solver& S, bool with_dot) {
  Reducer red = S.reducer(FIN_STORE);
  if (S.batch) {
    const Batch& B = *S.batch;
    if (S.mixed) k_seg_replace<LQ_F32><<<B.seg_grid, kBlas, 0, S.s>>>(S.rhi, S.r, S.Ap, B.seg, red, S.sc);
    else k_seg_replace<LQ_F64><<<B.seg_grid, kBlas, 0, S.s>>>(S.rhi, S.r, S.Ap, B.seg, red, S.sc);
    LQ_CHECK_LAUNCH(S.ctx, "k_seg_replace");
    return LQ_OK;
  }
  dim3 grid(S.nbx, S.nrhs);
  const CGScalars* sc = S.sc;
  if (S.paired) {
    // In the canonical layout, in x_lo (zero after the fold that precedes every
    // replacement, free until the next iteration) and t: r_old and Ap in, r_new out, then
    // back to the paired r; x_lo = 0 again.
    lq_status st;
    if (with_dot) {
      st = lq_vec_unpair(S.ctx, S.Vh, S.nrhs, S.r, S.xl, S.s);
      if (st) return st;
      st = lq_vec_unpair(S.ctx, S.Vh, S.nrhs, S.Ap, S.t, S.s);
      if (st) return st;
    }
    k_cg_replace<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.rhi, S.xl, S.t, sc, S.Vh, with_dot ? 1 : 0, red);
    LQ_CHECK_LAUNCH(S.ctx, "k_cg_replace");
    st = lq_vec_pair(S.ctx, S.Vh, S.nrhs, S.xl, S.r, S.s);
    if (st) return st;
    LQ_CUDA(S.ctx, cudaMemsetAsync(S.xl, 0, S.vin_bytes(), S.s));
    return LQ_OK;
  }
  if (S.mixed) k_cg_replace<LQ_F32><<<grid, kBlas, 0, S.s>>>(S.rhi, S.r, S.Ap, sc, S.Vh, with_dot ? 1 : 0, red);
  else k_cg_replace<LQ_F64><<<grid, kBlas, 0, S.s>>>(S.rhi, S.r, S.Ap, sc, S.Vh, with_dot ? 1 : 0, red);
  LQ_CHECK_LAUNCH(S.ctx, "k_cg_replace");
  return LQ_OK;
}

// r_hi = b with ||b||^2 -> result.
lq_status copy_source(Solver& S) {
  Reducer red = S.reducer(FIN_STORE);
  if (S.batch) {
    k_seg_convert<LQ_F64, LQ_F64><<<S.batch->seg_grid, kBlas, 0, S.s>>>(S.b, S.rhi, S.batch->seg, red, nullptr);
    LQ_CHECK_LAUNCH(S.ctx, "k_seg_convert(b)");
    return LQ_OK;
  }
  dim3 grid(S.nbx, S.nrhs);
  k_convert<LQ_F64, LQ_F64><<<grid, kBlas, 0, S.s>>>(S.b, S.rhi, S.Vh, 1, red);
  LQ_CHECK_LAUNCH(S.ctx, "k_convert(b)");
  return LQ_OK;
}

lq_status sync_scalars(Solver& S) {
  LQ_CUDA(S.ctx, cudaMemcpyAsync(S.sc_host, S.sc, sizeof(CGScalars) * S.nsys, cudaMemcpyDeviceToHost, S.s));
  LQ_CUDA(S.ctx, cudaStreamSynchronize(S.s));
  return LQ_OK;
}

lq_status push_scalars(Solver& S) {
  LQ_CUDA(S.ctx, cudaMemcpyAsync(S.sc, S.sc_host, sizeof(CGScalars) * S.nsys, cudaMemcpyHostToDevice, S.s));
  return LQ_OK;
}

// The first `rows` (default: one per system) FIN_STORE totals.
lq_status read_result(Solver& S, std::vector<double>& out, int rows = 0) {
  const int n = rows ? rows : S.nsys;
  out.resize(n);
  LQ_CUDA(S.ctx, cudaMemcpyAsync(out.data(), S.result, sizeof(double) * n, cudaMemcpyDeviceToHost, S.s));
  LQ_CUDA(S.ctx, cudaStreamSynchronize(S.s));
  return LQ_OK;
}

// After a solve: a bounded device wait that gave up since the context's status word was
// last reported (during the solve: the link-staging Dslash, whose block then skipped its
// work) invalidates the result: report LQ_ERR_TIMEOUT and clear the flag.
lq_status solve_status(lq_context* ctx, cudaStream_t s) {
  unsigned int flags = 0;
  LQ_CUDA(ctx, cudaMemcpyAsync(&flags, ctx->dev_status, sizeof flags, cudaMemcpyDeviceToHost, s));
  LQ_CUDA(ctx, cudaStreamSynchronize(s));
  if (!flags) return LQ_OK;
  LQ_CUDA(ctx, cudaMemsetAsync(ctx->dev_status, 0, sizeof flags, s));
  return lq_fail(ctx, LQ_ERR_TIMEOUT, "a bounded device wait gave up (status flags 0x%x) during the solve or "
                                      "before it, unreported: the solution is not valid", flags);
}

lq_status work_stream(lq_context* ctx, cudaStream_t* out) {
  static thread_local cudaStream_t cache[64] = {};
  int dev = ctx->device;
  if (dev < 0 || dev >= 64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "device index");
  if (!cache[dev]) LQ_CUDA(ctx, cudaStreamCreateWithFlags(&cache[dev], cudaStreamNonBlocking));
  *out = cache[dev];
  return LQ_OK;
}

// Pinned host copy of the per-system scalars (grown on demand).
lq_status host_scalars(lq_context* ctx, int nsys) {
  const size_t want = sizeof(CGScalars) * (nsys > 16 ? nsys : 16);
  if (ctx->host_pinned_bytes < want) {
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    LQ_CUDA(ctx, cudaMallocHost(&ctx->host_pinned, want));
    ctx->host_pinned_bytes = want;
  }
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
  const int n = S.nsys;
  const double tol2 = P.tol * P.tol;
  std::vector<double> res;
  std::vector<int> done(n, 0), updates(n, 0);
  std::vector<double> final_r2(n, 0.0);  // FP64 true residual^2 of each system once done
  std::vector<double> bb(n);
  lq_status st;

  // ---- initial state: x = 0, r = p = 0, r_hi = b, r = round(b), rr = ||r||^2
  LQ_CUDA(ctx, cudaMemsetAsync(S.x, 0, S.vbytes(LQ_F64), S.s));
  if (S.mixed) LQ_CUDA(ctx, cudaMemsetAsync(S.xl, 0, S.vin_bytes(), S.s));
  LQ_CUDA(ctx, cudaMemsetAsync(S.p, 0, S.vin_bytes(), S.s));
  st = copy_source(S);
  if (st) return st;
  st = read_result(S, res);
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    bb[i] = res[i];
    if (!isfinite(bb[i])) return lq_fail(ctx, LQ_ERR_NUMERIC, "source %d holds NaN/Inf", i);
  }
  // r = round(b) for every system (the batched kernel replaces the systems flagged ru)
  for (int i = 0; i < n; ++i) {
    memset(&S.sc_host[i], 0, sizeof(CGScalars));
    S.sc_host[i].ru = 1;
  }
  st = push_scalars(S);
  if (st) return st;
  st = replace_residual(S, /*with_dot=*/false);
  if (st) return st;
  st = read_result(S, res, 2 * n);
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    CGScalars& c = S.sc_host[i];
    memset(&c, 0, sizeof c);
    c.rr = res[2 * i];
    c.bb = bb[i];
    c.tol2 = tol2 * bb[i];
    c.rhi2 = bb[i];
    c.beta = 0.0;           // first xpay: p = r
    c.active = bb[i] > 0.0;
    if (bb[i] == 0.0) done[i] = c.done = 1;  // x = 0 solves it exactly
  }
  st = push_scalars(S);
  if (st) return st;

  GraphHolder graph;
  const int block = P.check_every > 0 ? P.check_every : 20;
  int total = 0, restarts_left = 8;
  std::vector<int> since(n, 0);   // inner iterations since each system's last reliable update
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
      for (int i = 0; i < n; ++i) since[i] += block;
      st = sync_scalars(S);
      if (st) return st;
    }
    // ---- decide on reliable updates, system by system
    std::vector<int> due(n, 0);
    bool need = false;
    for (int i = 0; i < n; ++i) {
      const CGScalars& c = S.sc_host[i];
      if (!isfinite(c.rr)) return lq_fail(ctx, LQ_ERR_NUMERIC, "residual of rhs %d became NaN/Inf", i);
      if (done[i]) continue;
      if (!c.active) due[i] = 1;  // apparent convergence: verify in FP64
      if (S.mixed && (since[i] >= P.reliable_every || c.rr < P.delta * P.delta * c.rhi2)) due[i] = 1;
      need |= due[i] != 0;
    }
    if (!need) continue;
    // The right-hand sides of one lattice take the update together, as in a single-lattice
    // solve (where one FP64 launch computes them all anyway); updating only the systems
    // whose own trigger fired was measured to stall BF16 inner solves, which rely on the
    // updates the other right-hand sides set off.  A batched solve leaves the lattices
    // without a due system alone: its FP64 launches skip their tiles (SKIP_NO_RU) and the
    // replacement does not touch their iteration.
    {
      const int nlat = S.batch ? S.batch->nlat : 1;
      const int per = n / nlat;   // systems are (lattice, rhs), lattice-major
      for (int l = 0; l < nlat; ++l) {
        bool any = false;
        for (int k = 0; k < per; ++k) any |= due[l * per + k] != 0;
        for (int k = 0; k < per; ++k) due[l * per + k] = any && !done[l * per + k];
      }
    }
    for (int i = 0; i < n; ++i) S.sc_host[i].ru = due[i];
    if (S.batch) {
      st = push_scalars(S);
      if (st) return st;
    }
    st = fold_x(S);              // exact for every system: x_hi + x_lo keeps its value
    if (st) return st;
    st = true_residual(S, S.batch ? SKIP_NO_RU : SKIP_DONE);
    if (st) return st;
    std::vector<double> rhi2;
    st = read_result(S, rhi2);
    if (st) return st;
    st = replace_residual(S, /*with_dot=*/true);
    if (st) return st;
    std::vector<double> rlo;   // [2 i]: ||r_lo||^2, [2 i + 1]: Re<r_lo, r_k>
    st = read_result(S, rlo, 2 * n);
    if (st) return st;
    bool restarted = false;
    for (int i = 0; i < n; ++i) {
      CGScalars& c = S.sc_host[i];
      c.ru = 0;
      if (done[i]) { c.active = 0; continue; }
      if (!due[i]) continue;
      since[i] = 0;
      updates[i] += 1;
      if (!isfinite(rhi2[i])) return lq_fail(ctx, LQ_ERR_NUMERIC, "true residual of rhs %d is NaN/Inf", i);
      if (rhi2[i] <= tol2 * bb[i]) {
        done[i] = 1;
        c.done = 1;
        c.active = 0;
        final_r2[i] = rhi2[i];
        continue;
      }
      if (!c.active) restarted = true;
      c.rhi2 = rhi2[i];
      const double pr = c.rr_prev > 0.0 ? (rlo[2 * i] - rlo[2 * i + 1]) / c.rr_prev : 0.0;
      c.beta = pr > 0.0 ? pr : 0.0;
      c.rr = rlo[2 * i];
      c.active = 1;
    }
    if (restarted && !S.mixed && --restarts_left < 0) break;
    st = push_scalars(S);
    if (st) return st;
  }
  // ---- final true residuals: a done system's x has not changed since its last FP64 check,
  // so the residual of that check stands; the others are recomputed.
  bool all_done = true;
  for (int i = 0; i < n; ++i) all_done &= done[i] != 0;
  if (all_done) {
    res = final_r2;
  } else {
    st = fold_x(S);
    if (st) return st;
    st = true_residual(S);
    if (st) return st;
    st = read_result(S, res);
    if (st) return st;
  }
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
  S.pdl = true;
  S.vp = S.mixed ? LQ_F32 : LQ_F64;
  S.mass = mass;
  S.nrhs = nrhs;
  S.Vh = U_hi->Vh;
  S.b = (const double*)b;
  S.x = (double*)x;
  S.nsys = nrhs;
  S.sites = (size_t)nrhs * S.Vh;
  S.nbx = (S.Vh + kBlas - 1) / kBlas;
  if (S.nbx > 8 * ctx->num_sms) S.nbx = 8 * ctx->num_sms;
  S.nblocks_max = (S.Vh + 15) / 16;  // Dslash reductions: up to 4 threads per site, blocks of 64
  if (S.nblocks_max < S.nbx) S.nblocks_max = S.nbx;
  // Two or more right-hand sides with reduced-precision links iterate on the paired
  // colour-planar layout (the environment variable LQCD_CG_PAIRED=0 keeps the canonical one)
  {
    const char* e = getenv("LQCD_CG_PAIRED");
    S.paired = S.mixed && nrhs >= 2 && S.Ulo->prec != LQ_F64 && !(e && e[0] == '0');
  }

  const size_t vin = S.vin_bytes(), v64 = S.vbytes(LQ_F64);
  const size_t need = 5 * vin + 2 * v64 + nrhs * (sizeof(CGScalars) + 16) + 8 +
                      3 * (size_t)nrhs * S.nblocks_max * sizeof(double) + (size_t)nrhs * kPapGroups * sizeof(double) +
                      14 * 256;
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
  S.result = (double*)A.take(sizeof(double) * 2 * nrhs);
  S.counter = (unsigned int*)A.take(sizeof(unsigned int));
  S.partials = (double*)A.take(sizeof(double) * 2 * nrhs * S.nblocks_max);
  S.dpartials = (double*)A.take(sizeof(double) * nrhs * S.nblocks_max);
  S.gsum = (double*)A.take(sizeof(double) * nrhs * kPapGroups);
  if (A.off > need) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "internal: scratch layout overflow");
  st = host_scalars(ctx, nrhs);
  if (st) return st;
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
  if (!st) st = solve_status(ctx, S.s);
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
  S.nsys = nrhs;
  S.sites = (size_t)nrhs * S.Vh;
  S.nbx = (S.Vh + kBlas - 1) / kBlas;
  if (S.nbx > 8 * ctx->num_sms) S.nbx = 8 * ctx->num_sms;
  S.nblocks_max = (S.Vh + 15) / 16;  // Dslash reductions: up to 4 threads per site, blocks of 64
  if (S.nblocks_max < S.nbx) S.nblocks_max = S.nbx;
  const size_t vin = S.vbytes(S.vp), v64 = S.vbytes(LQ_F64);
  const size_t need = (S.mixed ? 5 : 4) * vin + 2 * v64 + nrhs * (sizeof(CGScalars) + 16) + 8 +
                      3 * (size_t)nrhs * S.nblocks_max * sizeof(double) + (size_t)nrhs * kPapGroups * sizeof(double) +
                      14 * 256;
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
  S.result = (double*)A.take(sizeof(double) * 2 * nrhs);
  S.counter = (unsigned int*)A.take(sizeof(unsigned int));
  S.partials = (double*)A.take(sizeof(double) * 2 * nrhs * S.nblocks_max);
  S.dpartials = (double*)A.take(sizeof(double) * nrhs * S.nblocks_max);
  S.gsum = (double*)A.take(sizeof(double) * nrhs * kPapGroups);
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
  if (!st) st = solve_status(ctx, S.s);
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < nrhs; ++i) stats[i].seconds = secs;
  if (st) return st;
  if (!converged) return lq_fail(ctx, LQ_ERR_NOT_CONVERGED, "CG did not reach tol %.3g within %d iterations",
                                 params->tol, params->maxiter);
  return LQ_OK;
}

// ------------------------------------------------------------------ batched solve -----

static const char* prec_str(lq_prec p) {
  return p == LQ_F64 ? "f64" : p == LQ_F32 ? "f32" : p == LQ_BF16 ? "bf16" : "f16";
}

extern "C" lq_status cg_solve_batched(lq_context* ctx, int nlat, const lq_gauge* const* U_hi,
                                      const lq_gauge* const* U_lo, const double* mass, const void* const* b,
                                      void* const* x, int nrhs, const lq_cg_params* params, lq_cg_stats* stats,
                                      lq_stream stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (nlat < 1 || nlat > kMaxLat) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nlat must be in [1, %d]", kMaxLat);
  if (!U_hi || !mass || !b || !x || !params) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "NULL array argument");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (!(params->tol > 0.0) || params->maxiter < 1 || params->check_every < 1 || params->reliable_every < 1 ||
      !(params->delta >= 0.0 && params->delta < 1.0))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "bad CG parameters");
  const bool mixed = U_lo != nullptr;
  for (int l = 0; l < nlat; ++l) {
    if (!U_hi[l] || U_hi[l]->prec != LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_hi[%d] must be an LQ_F64 gauge", l);
    if (U_hi[l]->recon != U_hi[0]->recon) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "all U_hi must share recon");
    if (mixed) {
      if (!U_lo[l] || U_lo[l]->prec == LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_lo[%d] must be a reduced-precision gauge", l);
      if (U_lo[l]->prec != U_lo[0]->prec || U_lo[l]->recon != U_lo[0]->recon)
        return lq_fail(ctx, LQ_ERR_INVALID_ARG, "all U_lo must share precision and recon");
      for (int i = 0; i < 4; ++i)
        if (U_lo[l]->dims[i] != U_hi[l]->dims[i]) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U_lo[%d] and U_hi[%d] differ", l, l);
    }
    if (!b[l] || !x[l] || !lq_aligned16(b[l]) || !lq_aligned16(x[l]) || b[l] == x[l])
      return lq_fail(ctx, LQ_ERR_INVALID_ARG, "b[%d], x[%d] must be distinct 16-byte aligned device pointers", l, l);
  }
  DeviceGuard dg(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->mu);

  Batch B;
  B.nlat = nlat;
  size_t total = 0;
  int vh_max = 0;
  std::string lats;
  for (int l = 0; l < nlat; ++l) {
    B.hi[l] = U_hi[l];
    B.lo[l] = mixed ? U_lo[l] : U_hi[l];
    B.mass[l] = mass[l];
    B.voff[l] = total;
    total += (size_t)nrhs * U_hi[l]->Vh;
    if (U_hi[l]->Vh > vh_max) vh_max = U_hi[l]->Vh;
    char d[64];
    snprintf(d, sizeof d, "%s%dx%dx%dx%d", l ? "," : "", U_hi[l]->dims[0], U_hi[l]->dims[1], U_hi[l]->dims[2],
             U_hi[l]->dims[3]);
    lats += d;
  }
  char key[512];
  snprintf(key, sizeof key, "dslash_multi g=%s/%d v=%s lats=%s nrhs=%d", prec_str(B.lo[0]->prec),
           (int)B.lo[0]->recon, mixed ? "f32" : "f64", lats.c_str(), nrhs);
  B.key_lo = key;
  snprintf(key, sizeof key, "dslash_multi g=f64/%d v=f64 lats=%s nrhs=%d", (int)B.hi[0]->recon, lats.c_str(), nrhs);
  B.key_hi = key;

  Solver S{};
  S.ctx = ctx;
  S.Uhi = U_hi[0];
  S.Ulo = B.lo[0];
  S.mixed = mixed;
  S.vp = mixed ? LQ_F32 : LQ_F64;
  S.nrhs = nrhs;
  S.Vh = vh_max;
  S.nsys = nlat * nrhs;
  S.sites = total;
  S.batch = &B;
  S.nblocks_max = (vh_max + 15) / 16;
  memset(&B.seg, 0, sizeof B.seg);
  B.seg.nlat = nlat;
  B.seg.nrhs = nrhs;
  B.seg.pstride = (size_t)S.nblocks_max;
  int tiles = 0;
  for (int l = 0; l < nlat; ++l) {
    B.seg.lat[l].voff = B.voff[l];
    B.seg.lat[l].Vh = U_hi[l]->Vh;
    B.seg.lat[l].tile0 = tiles;
    B.seg.lat[l].tps = (U_hi[l]->Vh + kBlas - 1) / kBlas;
    tiles += nrhs * B.seg.lat[l].tps;
  }
  B.seg.ntiles = tiles;
  B.seg_grid = tiles < 8 * ctx->num_sms ? tiles : 8 * ctx->num_sms;

  const size_t vin = S.vbytes(S.vp), v64 = S.vbytes(LQ_F64);
  const size_t need = 5 * vin + 4 * v64 + S.nsys * (sizeof(CGScalars) + 16) + 8 +
                      3 * (size_t)S.nsys * S.nblocks_max * sizeof(double) + 15 * 256;
  void* base = nullptr;
  lq_status st = lq_scratch(ctx, need, &base);
  if (st) return st;
  Arena A{(char*)base};
  S.b = (const double*)A.take(v64);
  S.x = (double*)A.take(v64);
  S.xl = mixed ? A.take(vin) : (void*)S.x;
  S.r = A.take(vin);
  S.p = A.take(vin);
  S.Ap = A.take(vin);
  S.t = A.take(vin);
  S.rhi = (double*)A.take(v64);
  S.thi = (double*)A.take(v64);
  S.sc = (CGScalars*)A.take(sizeof(CGScalars) * S.nsys);
  S.result = (double*)A.take(sizeof(double) * 2 * S.nsys);
  S.counter = (unsigned int*)A.take(sizeof(unsigned int));
  S.partials = (double*)A.take(sizeof(double) * 2 * S.nsys * S.nblocks_max);
  S.dpartials = (double*)A.take(sizeof(double) * S.nsys * S.nblocks_max);
  if (A.off > need) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "internal: scratch layout overflow");
  st = host_scalars(ctx, S.nsys);
  if (st) return st;
  S.sc_host = (CGScalars*)ctx->host_pinned;

  cudaStream_t user = (cudaStream_t)stream;
  st = work_stream(ctx, &S.s);
  if (st) return st;
  cudaEvent_t ev;
  LQ_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  LQ_CUDA(ctx, cudaEventRecord(ev, user));
  LQ_CUDA(ctx, cudaStreamWaitEvent(S.s, ev, 0));
  LQ_CUDA(ctx, cudaMemsetAsync(S.counter, 0, sizeof(unsigned int), S.s));
  for (int l = 0; l < nlat; ++l)
    LQ_CUDA(ctx, cudaMemcpyAsync((char*)S.b + B.voff[l] * 48, b[l], (size_t)nrhs * U_hi[l]->Vh * 48,
                                 cudaMemcpyDeviceToDevice, S.s));
  int converged = 0;
  st = run_solver(S, *params, stats, &converged);
  if (!st) st = solve_status(ctx, S.s);
  if (!st)
    for (int l = 0; l < nlat && !st; ++l) {
      cudaError_t e = cudaMemcpyAsync(x[l], (const char*)S.x + B.voff[l] * 48, (size_t)nrhs * U_hi[l]->Vh * 48,
                                      cudaMemcpyDeviceToDevice, S.s);
      if (e != cudaSuccess) st = lq_cuda_fail(ctx, e, "copy of x");
    }
  cudaEventRecord(ev, S.s);
  cudaStreamWaitEvent(user, ev, 0);
  cudaEventDestroy(ev);
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < S.nsys; ++i) stats[i].seconds = secs;
  if (st) return st;
  if (!converged) return lq_fail(ctx, LQ_ERR_NOT_CONVERGED, "batched CG did not reach tol %.3g within %d iterations",
                                 params->tol, params->maxiter);
  return LQ_OK;
}
