// The half staggered Dslash kernel (one thread per output site and tile of right-hand
// sides) and its host-side launcher, instantiated per link storage format in
// dslash_<prec>.cu.
//
//   out(x) = c * sum_mu eta_mu(x) [ U_mu(x) in(x+mu) - U_mu(x-mu)^dag in(x-mu) ]
//            + a1 * w1(x) + a2 * w2(x)                      (x of parity out_parity)
//
// Forward hops are mult_su3_mat_vec summed over mu (mult_su3_mat_vec_sum_4dir of Table 1);
// backward hops are mult_adj_su3_mat_vec (Eqs. (1.1)-(2.3)), four per site
// (mult_adj_su3_mat_vec_4dir), combined as in sub_four_su3_vecs.  570 flops per site.
#pragma once

#include <string>
#include <vector>

#include "lqcd_internal.cuh"
#include "tune.cuh"

struct DslashKArgs {
  const char* gauge;
  size_t blk_bytes;
  Geom G;
  int out_par;
  const void* in;
  void* out;
  size_t rhs_stride;
  int nrhs;
  const void* w1;
  double a1;
  const void* w2;
  double a2;
  double c;
  int reduce;
  Reducer red;
};

template <lq_prec GP, int R, lq_prec VP, int NR>
__global__ void __launch_bounds__(256) k_dslash(const DslashKArgs a) {
  using L = LinkT<GP, R>;
  using VT = VecT<VP>;
  using T = typename L::real;
  const Geom G = a.G;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs0 = blockIdx.y * NR;
  const bool live = cb < G.Vh;
  double part[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) part[r] = 0.0;

  if (live) {
    // coordinates of the output site
    const int xh = cb % G.Lxh;
    const int row = cb / G.Lxh;         // y + Ly*(z + Lz*t)
    const int y = row % G.Ly;
    const int zt = row / G.Ly;
    const int z = zt % G.Lz;
    const int t = zt / G.Lz;
    const int x = 2 * xh + ((y + z + t + a.out_par) & 1);
    const int xf = (x + 1 == G.Lx) ? 0 : x + 1;
    const int xb = (x == 0) ? G.Lx - 1 : x - 1;
    const int sy = 1, sz = G.Ly, st = G.Ly * G.Lz;  // row strides
    const int rowf[4] = {row, (y + 1 == G.Ly) ? row - (G.Ly - 1) * sy : row + sy,
                         (z + 1 == G.Lz) ? row - (G.Lz - 1) * sz : row + sz,
                         (t + 1 == G.Lt) ? row - (G.Lt - 1) * st : row + st};
    const int rowb[4] = {row, (y == 0) ? row + (G.Ly - 1) * sy : row - sy,
                         (z == 0) ? row + (G.Lz - 1) * sz : row - sz,
                         (t == 0) ? row + (G.Lt - 1) * st : row - st};
    const T eta[4] = {T(1), (x & 1) ? T(-1) : T(1), ((x + y) & 1) ? T(-1) : T(1),
                      ((x + y + z) & 1) ? T(-1) : T(1)};

    T acc[NR][6];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[r][k] = T(0);

    const int opar = 1 - a.out_par;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int cbf = (mu == 0) ? (xf >> 1) + G.Lxh * row : xh + G.Lxh * rowf[mu];
      const int cbb = (mu == 0) ? (xb >> 1) + G.Lxh * row : xh + G.Lxh * rowb[mu];
      T u[18];
      // forward hop: U_mu(x) in(x+mu); U_mu(x) lives in block (mu, out_par) at cb
      L::load(a.gauge + (size_t)(2 * mu + a.out_par) * a.blk_bytes, G.S, cb, u);
      if (R == 12) reconstruct_row2(u);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (rhs0 + r < a.nrhs) {
          T v[6];
          VT::load(a.in, (size_t)(rhs0 + r) * a.rhs_stride + cbf, v);
          mat_vec_acc(u, v, acc[r], eta[mu]);
        }
      }
      // backward hop: U_mu(x-mu)^dag in(x-mu); that link lives in block (mu, 1-out_par)
      L::load(a.gauge + (size_t)(2 * mu + opar) * a.blk_bytes, G.S, cbb, u);
      if (R == 12) reconstruct_row2(u);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (rhs0 + r < a.nrhs) {
          T v[6];
          VT::load(a.in, (size_t)(rhs0 + r) * a.rhs_stride + cbb, v);
          adj_mat_vec_acc(u, v, acc[r], -eta[mu]);
        }
      }
    }

#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (rhs0 + r < a.nrhs) {
        const size_t site = (size_t)(rhs0 + r) * a.rhs_stride + cb;
        T res[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) res[k] = T(a.c) * acc[r][k];
        T w[6];
        if (a.w1) {
          VT::load(a.w1, site, w);
#pragma unroll
          for (int k = 0; k < 6; ++k) res[k] = fma(T(a.a1), w[k], res[k]);
        }
        if (a.w2) {
          T w2[6];
          VT::load(a.w2, site, w2);
#pragma unroll
          for (int k = 0; k < 6; ++k) res[k] = fma(T(a.a2), w2[k], res[k]);
        }
        VT::store(a.out, site, res);
        if (a.reduce == RED_DOT) {
          double d = 0.0;
#pragma unroll
          for (int k = 0; k < 6; ++k) d += (double)w[k] * (double)res[k];
          part[r] = d;
        } else if (a.reduce == RED_NORM) {
          double d = 0.0;
#pragma unroll
          for (int k = 0; k < 6; ++k) d += (double)res[k] * (double)res[k];
          part[r] = d;
        }
      }
    }
  }
  if (a.reduce != RED_NONE) block_reduce<NR>(part, a.red, rhs0, a.nrhs);
}

// Host side: launch one instance.
template <lq_prec GP, int R, lq_prec VP, int NR>
static cudaError_t launch_dslash_inst(const DslashKArgs& k, int block, cudaStream_t s) {
  dim3 grid((k.G.Vh + block - 1) / block, (k.nrhs + NR - 1) / NR);
  k_dslash<GP, R, VP, NR><<<grid, block, 0, s>>>(k);
  return cudaGetLastError();
}

template <lq_prec GP, int R, lq_prec VP>
static cudaError_t launch_dslash_tile(const DslashKArgs& k, int block, int tile, cudaStream_t s) {
  switch (tile) {
    case 1: return launch_dslash_inst<GP, R, VP, 1>(k, block, s);
    case 2: return launch_dslash_inst<GP, R, VP, 2>(k, block, s);
    case 4: return launch_dslash_inst<GP, R, VP, 4>(k, block, s);
    default: return launch_dslash_inst<GP, R, VP, 8>(k, block, s);
  }
}

// Entry used by dslash.cu for a given link storage format.
using DslashLaunchFn = cudaError_t (*)(const DslashKArgs&, lq_prec vec_prec, int block, int tile, cudaStream_t);

template <lq_prec GP, int R>
cudaError_t dslash_launch_gauge(const DslashKArgs& k, lq_prec vp, int block, int tile, cudaStream_t s) {
  if constexpr (GP == LQ_F64) {
    if (vp != LQ_F64) return cudaErrorInvalidValue;
    return launch_dslash_tile<GP, R, LQ_F64>(k, block, tile, s);
  } else {
    switch (vp) {
      case LQ_F32: return launch_dslash_tile<GP, R, LQ_F32>(k, block, tile, s);
      case LQ_BF16: return launch_dslash_tile<GP, R, LQ_BF16>(k, block, tile, s);
      case LQ_F16: return launch_dslash_tile<GP, R, LQ_F16>(k, block, tile, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

// Defined in the per-precision translation units.
DslashLaunchFn dslash_fn_f64(int recon);
DslashLaunchFn dslash_fn_f32(int recon);
DslashLaunchFn dslash_fn_bf16(int recon);
DslashLaunchFn dslash_fn_f16(int recon);
