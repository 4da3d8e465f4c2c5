// The single-lattice half staggered Dslash kernel and its host-side launcher,
// instantiated per link storage format in dslash_<prec>.cu.  The per-site arithmetic is
// in dslash_site.cuh.
#pragma once

#include <string>
#include <type_traits>
#include <vector>

#include "dslash_args.cuh"
#include "dslash_rw.cuh"
#include "dslash_site.cuh"
#include "dslash_tma.cuh"
#include "lqcd_internal.cuh"
#include "tune.cuh"

// One thread per (output site, direction group), TPS threads per site, NR right-hand sides
// per thread.  The rhs tiles of one block of sites are consecutive blocks of the grid
// (block b: rhs tile b % ntiles_y, site block b / ntiles_y), so they are dispatched
// together and read the same links while those are still in L2.
template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
__global__ void __launch_bounds__(256) k_dslash(const DslashKArgs a) {
  using T = typename LinkT<GP, R>::real;
  static_assert(TPS == 1 || TPS == 2 || TPS == 4, "TPS must be 1, 2 or 4");
  const int nty = (a.nrhs + NR - 1) / NR;
  const int ty = blockIdx.x % nty;
  const int bx = blockIdx.x / nty;
  const int gtid = bx * blockDim.x + threadIdx.x;
  const int cb = gtid / TPS;
  const int sub = gtid % TPS;
  const int rhs0 = ty * NR;
  const bool live = cb < a.G.Vh;
  // The thread's share of a fused reduction: FP32 (summed per warp by the compensated
  // FP32 tree) in the 12-real FP32 kernels, FP64 in the others.  Measured: with FP32
  // partials the plain 18-real FP32 operator, which never runs the reduction, went from
  // 5.58 to 5.87 us per 16^3 x 32 launch (the code around it changed, not the registers).
  using PT = typename std::conditional<R == 18, double, T>::type;
  PT part[NR];
  T acc[NR][6];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    part[r] = PT(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[r][k] = T(0);
  }
  pdl_wait();
  if (live)
    dslash_hops<GP, R, VP, NR, TPS>(a.gauge, a.blk_bytes, a.G, a.out_par, a.in, a.rhs_stride, a.nrhs, rhs0,
                                    cb, sub, acc);
  dslash_combine<NR, TPS>(acc);
  if (live)
    dslash_epilogue<VP, NR, TPS>(acc, a.out, a.w1, a.a1, a.w2, a.a2, a.c, a.reduce, a.rhs_stride, a.nrhs,
                                 rhs0, cb, sub, part);
  pdl_trigger();  // this block's main work is done: the successor may be scheduled
  // The compiler sizes and schedules the whole kernel with the finisher in it.  Measured:
  // with 12-real links the whole-block finisher raised the plain operator from 48 to 58
  // registers; with 18-real links the one-warp finisher slowed it (13.7 -> 17.4 us for a
  // lone 16^3 x 32 FP32 launch).  Each format keeps the finisher it runs fastest with.
  if (a.reduce != RED_NONE) block_reduce<NR, R == 18>(part, a.red, rhs0, a.nrhs, bx, gridDim.x / nty);
}

// Host side: launch one instance.  Supported (rhs tile, threads per site) pairs:
// (1|2, 1|2|4), (4, 1|2), (8, 1), and (RT x NRT, kTpsRhsWarps) for k_dslash_rw;
// dslash_shape_ok() (and dslash_rw_shape_ok()) tell the tuner.
inline bool dslash_shape_ok(int tile, int tps) {
  if (tps == kTpsRhsWarps) return tile >= 2 && tile <= 16;   // with the block: dslash_rw_shape_ok
  if (tps == kTpsTma) return tile == 1;                        // block from the geometry
  if (tile == 1 || tile == 2) return tps == 1 || tps == 2 || tps == 4;
  if (tile == 4) return tps == 1 || tps == 2;
  return tile == 8 && tps == 1;
}

template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
static cudaError_t launch_dslash_inst(const DslashKArgs& k, int block, cudaStream_t s) {
  const long long nbx = ((long long)k.G.Vh * TPS + block - 1) / block;
  dim3 grid((unsigned)(nbx * ((k.nrhs + NR - 1) / NR)));
  return launch_k(k_dslash<GP, R, VP, NR, TPS>, grid, dim3(block), 0, s, k.pdl != 0, k);
}

template <lq_prec GP, int R, lq_prec VP>
static cudaError_t launch_dslash_shape(const DslashKArgs& k, int block, int tile, int tps, cudaStream_t s) {
  if (tps == kTpsTma) return launch_dslash_tma<GP, R, VP>(k, s);
  if (tps == kTpsRhsWarps) {
    if constexpr (GP != LQ_F64 && VP == LQ_F32) {
      if (k.reduce != RED_NONE && k.red.finisher != FIN_DEFER) return cudaErrorInvalidValue;
      return launch_dslash_rw<GP, R>(k, block, tile, s);
    } else {
      return cudaErrorInvalidValue;
    }
  }
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

// Sites per block of the link-staging kernel for a gauge (0: not applicable).
template <lq_prec GP, int R>
int dslash_tma_block_of(const Geom& G) { return dslash_tma_block<GP, R>(G); }
using DslashTmaBlockFn = int (*)(const Geom&);

// Defined in the per-precision translation units.
DslashTmaBlockFn dslash_tma_fn_f32(int recon);
DslashTmaBlockFn dslash_tma_fn_bf16(int recon);
DslashTmaBlockFn dslash_tma_fn_f16(int recon);
DslashLaunchFn dslash_fn_f64(int recon);
DslashLaunchFn dslash_fn_f32(int recon);
DslashLaunchFn dslash_fn_bf16(int recon);
DslashLaunchFn dslash_fn_f16(int recon);
