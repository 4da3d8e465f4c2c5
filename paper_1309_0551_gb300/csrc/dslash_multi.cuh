// Multi-lattice half Dslash: one persistent launch applies the half Dslash to up to
// kMaxLat lattices of different sizes, each with nrhs right-hand sides ([nrhs][Vh_l][3]
// vectors per lattice).  The work is cut into tiles (lattice, block of sites, rhs tile --
// the rhs tiles of a site block adjacent, so they share its links in L2);
// a grid of about one wave of resident blocks walks the tiles in a fixed order (no queue,
// no waiting), so small lattices and the tail of large ones share the GPU.
#pragma once

#include "dslash_rw.cuh"
#include "dslash_site.cuh"
#include "tune.cuh"

constexpr int kMaxLat = 16;
constexpr int kMaxRows = kMaxLat * 16;   // (lattice, rhs) systems of one launch
enum { SKIP_INACTIVE = 1, SKIP_DONE = 2, SKIP_NO_RU = 3 };

// A system is skipped when it is inactive (SKIP_INACTIVE), done (SKIP_DONE), or does not
// take the reliable update under way (SKIP_NO_RU).
__device__ __forceinline__ bool system_skipped(const CGScalars& c, int mode) {
  return mode == SKIP_DONE ? c.done != 0 : mode == SKIP_NO_RU ? c.ru == 0 : c.active == 0;
}

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
  int skip_mode;                // skipped (system_skipped) are not computed
  Reducer red;        // rows q = l * nrhs + rhs; columns: the launch's blocks
  int* cols_out;      // host: receives the launch's block count (partial columns per row)
  MLat lat[kMaxLat];
};

// Reductions of the persistent kernels: each block adds its tiles' sums per row in shared
// memory (one writer per row: deterministic), then stores them as column blockIdx.x of
// partials[row][pstride] for every row; unless the finisher is deferred (FIN_DEFER: a later
// launch sums the rows), the last block sums the rows and runs the finisher.
__device__ __forceinline__ void multi_rows_init(double* sRow, int nrows) {
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) sRow[i] = 0.0;
  __syncthreads();
}
__device__ __forceinline__ void multi_rows_finish(const MultiKArgs& a, const double* sRow, int nrows) {
  __syncthreads();
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) a.red.partials[(size_t)i * a.pstride + blockIdx.x] = sRow[i];
  if (a.red.finisher != FIN_DEFER) grid_finish(a.red, nrows, a.pstride, [&](int) { return (int)gridDim.x; });
}

template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
__global__ void __launch_bounds__(256) k_dslash_multi(const MultiKArgs a) {
  using T = typename LinkT<GP, R>::real;
  using VT = VecT<VP>;
  __shared__ double sRow[kMaxRows];
  const int nrows = a.nlat * a.nrhs;
  if (a.reduce != RED_NONE) multi_rows_init(sRow, nrows);
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
        skip &= system_skipped(c, a.skip_mode);
      }
    }
    T part[NR];   // FP32 kernels: summed per warp by the compensated FP32 tree
#pragma unroll
    for (int r = 0; r < NR; ++r) part[r] = T(0);
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
      block_sum_add<NR>(part, sRow + l * a.nrhs + rhs0, nvalid);
    }
  }
  if (a.reduce != RED_NONE) multi_rows_finish(a, sRow, nrows);
}

// The multi-lattice form of the rhs-per-warp kernel (k_dslash_rw): a tile is (lattice,
// 32 sites, RT*NRT right-hand sides); a block of 32 x RT threads walks the tiles.  Per tile,
// warp w loads and rebuilds the links of hop w (w + RT, ...) into shared memory, then each
// thread applies them to its NRT right-hand sides of one site.  A reduction needs no block
// sum: every warp owns its right-hand sides, so each warp stores its own partials (column
// = the tile's site block).  FP32 vectors.
template <lq_prec GP, int R, int RT, int NRT>
__global__ void __launch_bounds__(32 * RT) k_dslash_multi_rw(const MultiKArgs a) {
  using L = LinkT<GP, R>;
  using VT = VecT<LQ_F32>;
  __shared__ float2 sU[8][9][32];
  __shared__ int sN[8][32];
  __shared__ double sRow[kMaxRows];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // 1-D block of 32 x RT threads
  constexpr int TR = RT * NRT;                // right-hand sides per tile
  const int nty = (a.nrhs + TR - 1) / TR;
  const int nrows = a.nlat * a.nrhs;
  if (a.reduce != RED_NONE) multi_rows_init(sRow, nrows);
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    int l = 0;
    while (l + 1 < a.nlat && tile >= a.lat[l + 1].tile0) ++l;
    const MLat& Lt = a.lat[l];
    const Geom& G = Lt.G;
    const int tl = tile - Lt.tile0;
    const int ty = tl % nty, tx = tl / nty;
    const int rhs0 = ty * TR + w * NRT;       // this warp's first right-hand side
    bool skip = false;                        // uniform over the block: the whole tile
    if (a.skip_state) {
      skip = true;
      for (int r = ty * TR; r < ty * TR + TR && r < a.nrhs; ++r) {
        const CGScalars& c = a.skip_state[l * a.nrhs + r];
        skip &= system_skipped(c, a.skip_mode);
      }
    }
    const int cb = tx * 32 + lane;
    float part[NRT];   // summed per warp by the compensated FP32 tree (warp_sum)
#pragma unroll
    for (int r = 0; r < NRT; ++r) part[r] = 0.f;
    if (!skip) {
      const int cbc = cb < G.Vh ? cb : G.Vh - 1;
      int xh, row, x, y, z, t;
      cb_coords(G, cbc, a.out_par, xh, row, x, y, z, t);
      for (int h = w; h < 8; h += RT) {
        const int mu = h >> 1;
        const bool bwd = h & 1;
        int cbf, cbb;
        dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
        const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
        const float sg = ((ephase & 1) ? -1.f : 1.f) * (bwd ? -1.f : 1.f);
        float u[18];
        L::load(Lt.gauge + (size_t)(2 * mu + (bwd ? 1 - a.out_par : a.out_par)) * Lt.blk_bytes, G.S,
                bwd ? cbb : cbc, u);
        if (R == 12) reconstruct_row2(u);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float er = bwd ? u[6 * j + 2 * i] : u[6 * i + 2 * j];
            const float ei = bwd ? -u[6 * j + 2 * i + 1] : u[6 * i + 2 * j + 1];
            sU[h][3 * i + j][lane] = make_float2(sg * er, sg * ei);
          }
        sN[h][lane] = bwd ? cbb : cbf;
      }
      __syncthreads();
      if (rhs0 < a.nrhs) {
        float acc[NRT][6];
        size_t roff[NRT];
#pragma unroll
        for (int r = 0; r < NRT; ++r) roff[r] = (size_t)min(rhs0 + r, a.nrhs - 1) * G.Vh;
        if constexpr (NRT == 1) {
          float v[8][6];
#pragma unroll
          for (int h = 0; h < 8; ++h) VT::load(Lt.in, roff[0] + sN[h][lane], v[h]);
#pragma unroll
          for (int k = 0; k < 6; ++k) acc[0][k] = 0.f;
#pragma unroll
          for (int h = 0; h < 8; ++h)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                const float2 e = sU[h][3 * i + j][lane];
                acc[0][2 * i] = fmaf(e.x, v[h][2 * j], acc[0][2 * i]);
                acc[0][2 * i] = fmaf(-e.y, v[h][2 * j + 1], acc[0][2 * i]);
                acc[0][2 * i + 1] = fmaf(e.x, v[h][2 * j + 1], acc[0][2 * i + 1]);
                acc[0][2 * i + 1] = fmaf(e.y, v[h][2 * j], acc[0][2 * i + 1]);
              }
        } else {
          float2 acc2[NRT / 2][6];
#pragma unroll
          for (int p = 0; p < NRT / 2; ++p)
#pragma unroll
            for (int k = 0; k < 6; ++k) acc2[p][k] = make_float2(0.f, 0.f);
          float v[2][NRT][6];
#pragma unroll
          for (int r = 0; r < NRT; ++r) VT::load(Lt.in, roff[r] + sN[0][lane], v[0][r]);
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const int cur = h & 1;
            if (h + 1 < 8) {
#pragma unroll
              for (int r = 0; r < NRT; ++r) VT::load(Lt.in, roff[r] + sN[h + 1][lane], v[cur ^ 1][r]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                const float2 e = sU[h][3 * i + j][lane];
                const float2 E = make_float2(e.x, e.x), F = make_float2(e.y, e.y), N = make_float2(-e.y, -e.y);
#pragma unroll
                for (int p = 0; p < NRT / 2; ++p) {
                  const float2 vr = make_float2(v[cur][2 * p][2 * j], v[cur][2 * p + 1][2 * j]);
                  const float2 vi = make_float2(v[cur][2 * p][2 * j + 1], v[cur][2 * p + 1][2 * j + 1]);
                  acc2[p][2 * i] = __ffma2_rn(E, vr, acc2[p][2 * i]);
                  acc2[p][2 * i] = __ffma2_rn(N, vi, acc2[p][2 * i]);
                  acc2[p][2 * i + 1] = __ffma2_rn(E, vi, acc2[p][2 * i + 1]);
                  acc2[p][2 * i + 1] = __ffma2_rn(F, vr, acc2[p][2 * i + 1]);
                }
              }
          }
#pragma unroll
          for (int p = 0; p < NRT / 2; ++p)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              acc[2 * p][k] = acc2[p][k].x;
              acc[2 * p + 1][k] = acc2[p][k].y;
            }
        }
        if (cb < G.Vh)
          dslash_epilogue<LQ_F32, NRT, 1>(acc, Lt.out, Lt.w1, Lt.a1, Lt.w2, Lt.a2, a.c, a.reduce, G.Vh, a.nrhs,
                                          rhs0, cb, 0, part);
      }
    }
    if (a.reduce != RED_NONE && rhs0 < a.nrhs) {
      // the warp owning rows rhs0 .. rhs0 + NRT - 1 of this lattice in every tile adds its sums
#pragma unroll
      for (int r = 0; r < NRT; ++r) {
        const double sum = warp_sum(part[r]);
        if (lane == 0 && rhs0 + r < a.nrhs) sRow[l * a.nrhs + rhs0 + r] += sum;
      }
    }
    __syncthreads();   // shared memory is rewritten by the next tile
  }
  if (a.reduce != RED_NONE) multi_rows_finish(a, sRow, nrows);
}

// Launch-shape helpers -----------------------------------------------------------------
inline bool dslash_multi_shape_ok(int tile, int tps) {
  if (tps == kTpsRhsWarps) return tile >= 2 && tile <= 16;   // with the block: dslash_rw_shape_ok
  return (tile == 1 || tile == 2 || tile == 4 || tile == 8) && (tps == 1 || tps == 2 || tps == 4);
}

// Fills the tile bookkeeping of `a` for a launch shape; returns the number of tiles.
inline int multi_tiles(MultiKArgs& a, int block, int tile, int tps) {
  int t0 = 0;
  const int ty = (a.nrhs + tile - 1) / tile;
  for (int l = 0; l < a.nlat; ++l) {
    a.lat[l].tile0 = t0;
    a.lat[l].tiles_x = tps == kTpsRhsWarps ? (a.lat[l].G.Vh + 31) / 32
                                           : (int)(((long long)a.lat[l].G.Vh * tps + block - 1) / block);
    t0 += a.lat[l].tiles_x * ty;
  }
  a.ntiles = t0;
  return t0;
}

template <lq_prec GP, int R, int RT, int NRT>
static cudaError_t launch_multi_rw_inst(MultiKArgs a, int num_sms, cudaStream_t s) {
  multi_tiles(a, 32 * RT, RT * NRT, kTpsRhsWarps);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash_multi_rw<GP, R, RT, NRT>, 32 * RT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (a.reduce != RED_NONE && (size_t)grid > a.pstride) grid = (int)a.pstride;
  if (grid < 1) return cudaSuccess;
  if (a.cols_out) *a.cols_out = grid;
  k_dslash_multi_rw<GP, R, RT, NRT><<<grid, 32 * RT, 0, s>>>(a);
  return cudaGetLastError();
}

template <lq_prec GP, int R>
static cudaError_t launch_multi_rw(const MultiKArgs& a, int block, int tile, int num_sms, cudaStream_t s) {
  if (!dslash_rw_shape_ok(block, tile)) return cudaErrorInvalidValue;
  const int rt = block / 32, nrt = tile / rt;
  switch (rt * 8 + nrt) {
    case 2 * 8 + 1: return launch_multi_rw_inst<GP, R, 2, 1>(a, num_sms, s);
    case 2 * 8 + 2: return launch_multi_rw_inst<GP, R, 2, 2>(a, num_sms, s);
    case 2 * 8 + 4: return launch_multi_rw_inst<GP, R, 2, 4>(a, num_sms, s);
    case 4 * 8 + 1: return launch_multi_rw_inst<GP, R, 4, 1>(a, num_sms, s);
    case 4 * 8 + 2: return launch_multi_rw_inst<GP, R, 4, 2>(a, num_sms, s);
    case 4 * 8 + 4: return launch_multi_rw_inst<GP, R, 4, 4>(a, num_sms, s);
    case 8 * 8 + 1: return launch_multi_rw_inst<GP, R, 8, 1>(a, num_sms, s);
    case 8 * 8 + 2: return launch_multi_rw_inst<GP, R, 8, 2>(a, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
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
  if (a.reduce != RED_NONE && (size_t)grid > a.pstride) grid = (int)a.pstride;
  if (grid < 1) return cudaSuccess;
  if (a.cols_out) *a.cols_out = grid;
  k_dslash_multi<GP, R, VP, NR, TPS><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <lq_prec GP, int R, lq_prec VP>
static cudaError_t launch_multi_shape(const MultiKArgs& a, int block, int tile, int tps, int num_sms, cudaStream_t s) {
  if (tps == kTpsRhsWarps) {
    if constexpr (GP != LQ_F64 && VP == LQ_F32) return launch_multi_rw<GP, R>(a, block, tile, num_sms, s);
    else return cudaErrorInvalidValue;
  }
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
