// Multi-lattice half Dslash: one persistent launch applies the half Dslash to up to
// kMaxLat lattices of different sizes, each with nrhs right-hand sides ([nrhs][Vh_l][3]
// vectors per lattice).  The work is cut into tiles (lattice, block of sites, rhs tile --
// the rhs tiles of a site block adjacent, so they share its links in L2);
// a grid of about one wave of resident blocks walks the tiles in a fixed order (no queue,
// no waiting), so small lattices and the tail of large ones share the GPU.
#pragma once

#include "dslash_site.cuh"
#include "tune.cuh"

constexpr int kMaxLat = 16;
enum { SKIP_INACTIVE = 1, SKIP_DONE = 2 };

struct MLat {
  const char* gauge;  // packed links of this lattice
  size_t blk_bytes;
  Geom G;
  const void* in;     // this lattice's vectors
  void* out;
  const void* w1;     // optional epilogue vectors
  const void* w2;
  double a1, a2;      // epilogue coefficients of this lattice
  int tile0;          // first tile of this lattice
  int tiles_x;        // site blocks per rhs tile
};

struct MultiKArgs {
  int nlat, ntiles, nrhs, out_par;
  double c;
  int reduce;
  size_t pstride;     // partials row stride (columns per (lattice, rhs) row)
  const CGScalars* skip_state;  // optional per-system state: tiles whose systems are all
  int skip_mode;                // inactive (SKIP_INACTIVE) or all done (SKIP_DONE) are skipped
  Reducer red;        // rows q = l * nrhs + rhs
  MLat lat[kMaxLat];
};

template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
__global__ void __launch_bounds__(256) k_dslash_multi(const MultiKArgs a) {
  using T = typename LinkT<GP, R>::real;
  using VT = VecT<VP>;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    int l = 0;
    while (l + 1 < a.nlat && tile >= a.lat[l + 1].tile0) ++l;
    const MLat& L = a.lat[l];
    const int tl = tile - L.tile0;
    const int nty = (a.nrhs + NR - 1) / NR;   // rhs tiles of one site block are adjacent
    const int ty = tl % nty, tx = tl / nty;
    const int rhs0 = ty * NR;
    bool skip = false;
    if (a.skip_state) {
      skip = true;
      for (int r = 0; r < NR && rhs0 + r < a.nrhs; ++r) {
        const CGScalars& c = a.skip_state[l * a.nrhs + rhs0 + r];
        skip &= (a.skip_mode == SKIP_DONE) ? (c.done != 0) : (c.active == 0);
      }
    }
    double part[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) part[r] = 0.0;
    if (!skip) {
      const int gtid = tx * blockDim.x + threadIdx.x;
      const int cb = gtid / TPS;
      const int sub = gtid % TPS;
      const bool live = cb < L.G.Vh;
      T acc[NR][6];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[r][k] = T(0);
      if (live)
        dslash_hops<GP, R, VP, NR, TPS>(L.gauge, L.blk_bytes, L.G, a.out_par, L.in, L.G.Vh, a.nrhs, rhs0, cb,
                                        sub, acc);
      dslash_combine<NR, TPS>(acc);
      if (live)
        dslash_epilogue<VP, NR, TPS>(acc, L.out, L.w1, L.a1, L.w2, L.a2, a.c, a.reduce, L.G.Vh, a.nrhs, rhs0, cb,
                                     sub, part);
    }
    if (a.reduce != RED_NONE) {
      const int nvalid = a.nrhs - rhs0 < NR ? a.nrhs - rhs0 : NR;
      block_sum_store<NR>(part, a.red.partials + (size_t)(l * a.nrhs + rhs0) * a.pstride + tx, a.pstride, nvalid);
    }
  }
  if (a.reduce != RED_NONE)
    grid_finish(a.red, a.nlat * a.nrhs, a.pstride, [&](int q) { return a.lat[q / a.nrhs].tiles_x; });
}

// Launch-shape helpers -----------------------------------------------------------------
inline bool dslash_multi_shape_ok(int tile, int tps) {
  return (tile == 1 || tile == 2 || tile == 4 || tile == 8) && (tps == 1 || tps == 2 || tps == 4);
}

// Fills the tile bookkeeping of `a` for a launch shape; returns the number of tiles.
inline int multi_tiles(MultiKArgs& a, int block, int tile, int tps) {
  int t0 = 0;
  const int ty = (a.nrhs + tile - 1) / tile;
  for (int l = 0; l < a.nlat; ++l) {
    a.lat[l].tile0 = t0;
    a.lat[l].tiles_x = (int)(((long long)a.lat[l].G.Vh * tps + block - 1) / block);
    t0 += a.lat[l].tiles_x * ty;
  }
  a.ntiles = t0;
  return t0;
}

template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
static cudaError_t launch_multi_inst(MultiKArgs a, int block, int num_sms, cudaStream_t s) {
  multi_tiles(a, block, NR, TPS);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash_multi<GP, R, VP, NR, TPS>, block, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) return cudaSuccess;
  k_dslash_multi<GP, R, VP, NR, TPS><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <lq_prec GP, int R, lq_prec VP>
static cudaError_t launch_multi_shape(const MultiKArgs& a, int block, int tile, int tps, int num_sms, cudaStream_t s) {
  switch (tile * 8 + tps) {
    case 1 * 8 + 1: return launch_multi_inst<GP, R, VP, 1, 1>(a, block, num_sms, s);
    case 1 * 8 + 2: return launch_multi_inst<GP, R, VP, 1, 2>(a, block, num_sms, s);
    case 1 * 8 + 4: return launch_multi_inst<GP, R, VP, 1, 4>(a, block, num_sms, s);
    case 2 * 8 + 1: return launch_multi_inst<GP, R, VP, 2, 1>(a, block, num_sms, s);
    case 2 * 8 + 2: return launch_multi_inst<GP, R, VP, 2, 2>(a, block, num_sms, s);
    case 2 * 8 + 4: return launch_multi_inst<GP, R, VP, 2, 4>(a, block, num_sms, s);
    case 4 * 8 + 1: return launch_multi_inst<GP, R, VP, 4, 1>(a, block, num_sms, s);
    case 4 * 8 + 2: return launch_multi_inst<GP, R, VP, 4, 2>(a, block, num_sms, s);
    case 4 * 8 + 4: return launch_multi_inst<GP, R, VP, 4, 4>(a, block, num_sms, s);
    case 8 * 8 + 1: return launch_multi_inst<GP, R, VP, 8, 1>(a, block, num_sms, s);
    case 8 * 8 + 2: return launch_multi_inst<GP, R, VP, 8, 2>(a, block, num_sms, s);
    case 8 * 8 + 4: return launch_multi_inst<GP, R, VP, 8, 4>(a, block, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

using MultiLaunchFn = cudaError_t (*)(const MultiKArgs&, lq_prec vec_prec, int block, int tile, int tps,
                                      int num_sms, cudaStream_t);

// FP64 links take FP64 vectors; the other formats take FP32 vectors (the solvers' inner
// precision).
template <lq_prec GP, int R>
cudaError_t multi_launch_gauge(const MultiKArgs& a, lq_prec vp, int block, int tile, int tps, int num_sms,
                               cudaStream_t s) {
  if constexpr (GP == LQ_F64) {
    if (vp != LQ_F64) return cudaErrorInvalidValue;
    return launch_multi_shape<GP, R, LQ_F64>(a, block, tile, tps, num_sms, s);
  } else {
    if (vp != LQ_F32) return cudaErrorInvalidValue;
    return launch_multi_shape<GP, R, LQ_F32>(a, block, tile, tps, num_sms, s);
  }
}

MultiLaunchFn dslash_multi_fn(lq_prec prec, int recon);
