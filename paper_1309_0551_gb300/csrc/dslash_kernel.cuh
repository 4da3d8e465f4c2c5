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

// TPS threads share one output site (TPS in {1, 2, 4}; consecutive lanes): thread `sub`
// applies the forward and backward hops of directions sub*(4/TPS) ... (sub+1)*(4/TPS)-1,
// the partial sums are combined with xor shuffles, and output colour component c is
// finished and stored by lane c % TPS.  More threads per site put more independent loads
// in flight when the lattice alone would leave the GPU under-occupied.
template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
__global__ void __launch_bounds__(256) k_dslash(const DslashKArgs a) {
  using L = LinkT<GP, R>;
  using VT = VecT<VP>;
  using T = typename L::real;
  static_assert(TPS == 1 || TPS == 2 || TPS == 4, "TPS must be 1, 2 or 4");
  constexpr int DPT = 4 / TPS;   // directions per thread
  const Geom G = a.G;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int cb = gtid / TPS;
  const int sub = gtid % TPS;
  const int rhs0 = blockIdx.y * NR;
  const bool live = cb < G.Vh;
  double part[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) part[r] = 0.0;

  T acc[NR][6];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[r][k] = T(0);

  // coordinates of the output site
  const int xh = cb % G.Lxh;
  const int row = cb / G.Lxh;         // y + Ly*(z + Lz*t)
  const int y = row % G.Ly;
  const int zt = row / G.Ly;
  const int z = zt % G.Lz;
  const int t = zt / G.Lz;
  const int x = 2 * xh + ((y + z + t + a.out_par) & 1);

  if (live) {
    const int opar = 1 - a.out_par;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int mu = sub * DPT + j;
      int cbf, cbb;
      if (mu == 0) {
        const int xf = (x + 1 == G.Lx) ? 0 : x + 1;
        const int xb = (x == 0) ? G.Lx - 1 : x - 1;
        cbf = (xf >> 1) + G.Lxh * row;
        cbb = (xb >> 1) + G.Lxh * row;
      } else {
        const int c = (mu == 1) ? y : (mu == 2) ? z : t;
        const int Lm = (mu == 1) ? G.Ly : (mu == 2) ? G.Lz : G.Lt;
        const int sm = (mu == 1) ? 1 : (mu == 2) ? G.Ly : G.Ly * G.Lz;   // row stride
        const int rf = (c + 1 == Lm) ? row - (Lm - 1) * sm : row + sm;
        const int rb = (c == 0) ? row + (Lm - 1) * sm : row - sm;
        cbf = xh + G.Lxh * rf;
        cbb = xh + G.Lxh * rb;
      }
      const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
      const T eta = (ephase & 1) ? T(-1) : T(1);
      T u[18];
      // forward hop: U_mu(x) in(x+mu); U_mu(x) lives in block (mu, out_par) at cb
      L::load(a.gauge + (size_t)(2 * mu + a.out_par) * a.blk_bytes, G.S, cb, u);
      if (R == 12) reconstruct_row2(u);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (rhs0 + r < a.nrhs) {
          T v[6];
          VT::load(a.in, (size_t)(rhs0 + r) * a.rhs_stride + cbf, v);
          mat_vec_acc(u, v, acc[r], eta);
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
          adj_mat_vec_acc(u, v, acc[r], -eta);
        }
      }
    }
  }

  // combine the TPS partial sums of a site (all lanes take part, dead ones add zeros)
#pragma unroll
  for (int off = 1; off < TPS; off <<= 1)
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[r][k] += __shfl_xor_sync(0xffffffffu, acc[r][k], off);

  if (live) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (rhs0 + r < a.nrhs) {
        const size_t site = (size_t)(rhs0 + r) * a.rhs_stride + cb;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (c % TPS != sub) continue;
          T res[2] = {T(a.c) * acc[r][2 * c], T(a.c) * acc[r][2 * c + 1]};
          T w[2] = {T(0), T(0)};
          if (a.w1) {
            VT::load_c(a.w1, site, c, w);
            res[0] = fma(T(a.a1), w[0], res[0]);
            res[1] = fma(T(a.a1), w[1], res[1]);
          }
          if (a.w2) {
            T w2[2];
            VT::load_c(a.w2, site, c, w2);
            res[0] = fma(T(a.a2), w2[0], res[0]);
            res[1] = fma(T(a.a2), w2[1], res[1]);
          }
          VT::store_c(a.out, site, c, res);
          if (a.reduce == RED_DOT)
            part[r] += (double)w[0] * (double)res[0] + (double)w[1] * (double)res[1];
          else if (a.reduce == RED_NORM)
            part[r] += (double)res[0] * (double)res[0] + (double)res[1] * (double)res[1];
        }
      }
    }
  }
  if (a.reduce != RED_NONE) block_reduce<NR>(part, a.red, rhs0, a.nrhs);
}

// Host side: launch one instance.  Supported (rhs tile, threads per site) pairs:
// (1|2, 1|2|4), (4, 1|2), (8, 1); dslash_shape_ok() tells the tuner.
inline bool dslash_shape_ok(int tile, int tps) {
  if (tile == 1 || tile == 2) return tps == 1 || tps == 2 || tps == 4;
  if (tile == 4) return tps == 1 || tps == 2;
  return tile == 8 && tps == 1;
}

template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
static cudaError_t launch_dslash_inst(const DslashKArgs& k, int block, cudaStream_t s) {
  dim3 grid((unsigned)(((long long)k.G.Vh * TPS + block - 1) / block), (k.nrhs + NR - 1) / NR);
  k_dslash<GP, R, VP, NR, TPS><<<grid, block, 0, s>>>(k);
  return cudaGetLastError();
}

template <lq_prec GP, int R, lq_prec VP>
static cudaError_t launch_dslash_shape(const DslashKArgs& k, int block, int tile, int tps, cudaStream_t s) {
  switch (tile * 8 + tps) {
    case 1 * 8 + 1: return launch_dslash_inst<GP, R, VP, 1, 1>(k, block, s);
    case 1 * 8 + 2: return launch_dslash_inst<GP, R, VP, 1, 2>(k, block, s);
    case 1 * 8 + 4: return launch_dslash_inst<GP, R, VP, 1, 4>(k, block, s);
    case 2 * 8 + 1: return launch_dslash_inst<GP, R, VP, 2, 1>(k, block, s);
    case 2 * 8 + 2: return launch_dslash_inst<GP, R, VP, 2, 2>(k, block, s);
    case 2 * 8 + 4: return launch_dslash_inst<GP, R, VP, 2, 4>(k, block, s);
    case 4 * 8 + 1: return launch_dslash_inst<GP, R, VP, 4, 1>(k, block, s);
    case 4 * 8 + 2: return launch_dslash_inst<GP, R, VP, 4, 2>(k, block, s);
    case 8 * 8 + 1: return launch_dslash_inst<GP, R, VP, 8, 1>(k, block, s);
    default: return cudaErrorInvalidValue;
  }
}

// Entry used by dslash.cu for a given link storage format.
using DslashLaunchFn = cudaError_t (*)(const DslashKArgs&, lq_prec vec_prec, int block, int tile, int tps,
                                       cudaStream_t);

template <lq_prec GP, int R>
cudaError_t dslash_launch_gauge(const DslashKArgs& k, lq_prec vp, int block, int tile, int tps, cudaStream_t s) {
  if constexpr (GP == LQ_F64) {
    if (vp != LQ_F64) return cudaErrorInvalidValue;
    return launch_dslash_shape<GP, R, LQ_F64>(k, block, tile, tps, s);
  } else {
    switch (vp) {
      case LQ_F32: return launch_dslash_shape<GP, R, LQ_F32>(k, block, tile, tps, s);
      case LQ_BF16: return launch_dslash_shape<GP, R, LQ_BF16>(k, block, tile, tps, s);
      case LQ_F16: return launch_dslash_shape<GP, R, LQ_F16>(k, block, tile, tps, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

// Defined in the per-precision translation units.
DslashLaunchFn dslash_fn_f64(int recon);
DslashLaunchFn dslash_fn_f32(int recon);
DslashLaunchFn dslash_fn_bf16(int recon);
DslashLaunchFn dslash_fn_f16(int recon);
