// Improved staggered half Dslash: one-hop ("fat") and three-hop ("long", Naik) links.
//
//   out(x) = sum_mu eta_mu(x) [ F_mu(x) in(x+mu)   - F_mu(x-mu)^dag  in(x-mu)
//                              + L_mu(x) in(x+3mu) - L_mu(x-3mu)^dag in(x-3mu) ]
//
// 16 hops per site: 1146 flops (16 mat-vecs of 66, 15 colour-vector sums of 6).  Both link
// fields use the 18-real layout of lq_gauge (fat links are not unitary; long links carry a
// coefficient).  Same thread layout as the plain kernel: TPS threads per site split the
// directions, NR right-hand sides per thread, rhs tiles of a site block adjacent.
#pragma once

#include "dslash_site.cuh"
#include "lqcd_internal.cuh"
#include "tune.cuh"

struct ImpKArgs {
  const char* fat;
  const char* lng;
  size_t blk_bytes;   // identical for both fields (same format and lattice)
  Geom G;
  int out_par;
  const void* in;
  void* out;
  size_t rhs_stride;
  int nrhs;
};

template <lq_prec GP, lq_prec VP, int NR, int TPS>
__global__ void __launch_bounds__(256) k_dslash_improved(const ImpKArgs a) {
  using L = LinkT<GP, 18>;
  using VT = VecT<VP>;
  using T = typename L::real;
  constexpr int DPT = 4 / TPS;
  const Geom G = a.G;
  const int nty = (a.nrhs + NR - 1) / NR;
  const int ty = blockIdx.x % nty;
  const int bx = blockIdx.x / nty;
  const int gtid = bx * blockDim.x + threadIdx.x;
  const int cb = gtid / TPS;
  const int sub = gtid % TPS;
  const int rhs0 = ty * NR;
  const bool live = cb < G.Vh;
  T acc[NR][6];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[r][k] = T(0);
  if (live) {
    int xh, row, x, y, z, t;
    cb_coords(G, cb, a.out_par, xh, row, x, y, z, t);
    const int opar = 1 - a.out_par;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int mu = sub * DPT + j;
      const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
      const T eta = (ephase & 1) ? T(-1) : T(1);
#pragma unroll
      for (int n = 1; n <= 3; n += 2) {   // one hop (fat links), three hops (long links)
        const char* field = (n == 1) ? a.fat : a.lng;
        int cbf, cbb;
        if (mu == 0) {
          const int xf = (x + n) % G.Lx;
          const int xb = (x - n + 3 * G.Lx) % G.Lx;
          cbf = (xf >> 1) + G.Lxh * row;
          cbb = (xb >> 1) + G.Lxh * row;
        } else {
          const int c = (mu == 1) ? y : (mu == 2) ? z : t;
          const int Lm = (mu == 1) ? G.Ly : (mu == 2) ? G.Lz : G.Lt;
          const int sm = (mu == 1) ? 1 : (mu == 2) ? G.Ly : G.Ly * G.Lz;
          const int cf = (c + n) % Lm;
          const int cbk = (c - n + 3 * Lm) % Lm;
          cbf = xh + G.Lxh * (row + (cf - c) * sm);
          cbb = xh + G.Lxh * (row + (cbk - c) * sm);
        }
        T u[18];
        // forward: W_mu(x) in(x+n mu), W_mu(x) in block (mu, out_par) at cb
        L::load(field + (size_t)(2 * mu + a.out_par) * a.blk_bytes, G.S, cb, u);
        {
          T v[NR][6];
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (rhs0 + r < a.nrhs) VT::load(a.in, (size_t)(rhs0 + r) * a.rhs_stride + cbf, v[r]);
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (rhs0 + r < a.nrhs) mat_vec_acc(u, v[r], acc[r], eta);
        }
        // backward: W_mu(x-n mu)^dag in(x-n mu); x - n mu has the other parity (n odd)
        L::load(field + (size_t)(2 * mu + opar) * a.blk_bytes, G.S, cbb, u);
        {
          T v[NR][6];
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (rhs0 + r < a.nrhs) VT::load(a.in, (size_t)(rhs0 + r) * a.rhs_stride + cbb, v[r]);
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (rhs0 + r < a.nrhs) adj_mat_vec_acc(u, v[r], acc[r], -eta);
        }
      }
    }
  }
  dslash_combine<NR, TPS>(acc);
  double part[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) part[r] = 0.0;
  if (live)
    dslash_epilogue<VP, NR, TPS>(acc, a.out, nullptr, 0.0, nullptr, 0.0, 1.0, RED_NONE, a.rhs_stride, a.nrhs, rhs0,
                                 cb, sub, part);
}

inline bool improved_shape_ok(int tile, int tps) {
  return (tile == 1 || tile == 2 || tile == 4) && (tps == 1 || tps == 2);
}

template <lq_prec GP, lq_prec VP, int NR, int TPS>
static cudaError_t launch_improved_inst(const ImpKArgs& k, int block, cudaStream_t s) {
  const long long nbx = ((long long)k.G.Vh * TPS + block - 1) / block;
  k_dslash_improved<GP, VP, NR, TPS><<<(unsigned)(nbx * ((k.nrhs + NR - 1) / NR)), block, 0, s>>>(k);
  return cudaGetLastError();
}

template <lq_prec GP, lq_prec VP>
static cudaError_t launch_improved_shape(const ImpKArgs& k, int block, int tile, int tps, cudaStream_t s) {
  switch (tile * 8 + tps) {
    case 1 * 8 + 1: return launch_improved_inst<GP, VP, 1, 1>(k, block, s);
    case 1 * 8 + 2: return launch_improved_inst<GP, VP, 1, 2>(k, block, s);
    case 2 * 8 + 1: return launch_improved_inst<GP, VP, 2, 1>(k, block, s);
    case 2 * 8 + 2: return launch_improved_inst<GP, VP, 2, 2>(k, block, s);
    case 4 * 8 + 1: return launch_improved_inst<GP, VP, 4, 1>(k, block, s);
    case 4 * 8 + 2: return launch_improved_inst<GP, VP, 4, 2>(k, block, s);
    default: return cudaErrorInvalidValue;
  }
}

using ImprovedLaunchFn = cudaError_t (*)(const ImpKArgs&, lq_prec vec_prec, int block, int tile, int tps,
                                         cudaStream_t);

template <lq_prec GP>
cudaError_t improved_launch_gauge(const ImpKArgs& k, lq_prec vp, int block, int tile, int tps, cudaStream_t s) {
  if constexpr (GP == LQ_F64) {
    if (vp != LQ_F64) return cudaErrorInvalidValue;
    return launch_improved_shape<GP, LQ_F64>(k, block, tile, tps, s);
  } else {
    switch (vp) {
      case LQ_F32: return launch_improved_shape<GP, LQ_F32>(k, block, tile, tps, s);
      case LQ_BF16: return launch_improved_shape<GP, LQ_BF16>(k, block, tile, tps, s);
      case LQ_F16: return launch_improved_shape<GP, LQ_F16>(k, block, tile, tps, s);
      default: return cudaErrorInvalidValue;
    }
  }
}
