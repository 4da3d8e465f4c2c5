// The single-lattice half staggered Dslash kernel and its host-side launcher,
// instantiated per link storage format in dslash_<prec>.cu.  The per-site arithmetic is
// in dslash_site.cuh.
#pragma once

#include <string>
#include <vector>

#include "dslash_site.cuh"
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
  int pdl;     // host side only: launch with programmatic dependent launch
};

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
  double part[NR];
  T acc[NR][6];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    part[r] = 0.0;
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
  if (a.reduce != RED_NONE) block_reduce<NR>(part, a.red, rhs0, a.nrhs, bx, gridDim.x / nty);
}

// Multi-RHS half Dslash with the right-hand sides spread over warps: a block holds 32
// sites (lanes) x RT warps, each thread NRT right-hand sides of one site.  Warp w loads the
// links of hop w (and w + RT, ...) for the block's 32 sites once, rebuilds them, folds in
// the hop's sign and writes op(U) (U_mu(x) forward, U_mu(x-mu)^dag backward) to shared
// memory with the neighbour index; after one barrier every thread applies the eight shared
// links to its right-hand sides.  Link loads and the 12-real reconstruction are done once
// per site and hop, not once per rhs; each link element read from shared memory serves
// NRT right-hand sides (in pairs, with packed FP32x2 FMAs, when NRT is even).
// FP32 vectors and arithmetic; no fused reduction (RED_NONE).
template <lq_prec GP, int R, int RT, int NRT>
__global__ void __launch_bounds__(32 * RT) k_dslash_rw(const DslashKArgs a) {
  using L = LinkT<GP, R>;
  using VT = VecT<LQ_F32>;
  __shared__ float2 sU[8][9][32];   // [hop][element 3i+j of op(U), sign folded][site]
  __shared__ int sN[8][32];         // [hop][site]: checkerboard index of the neighbour
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // 1-D block of 32 x RT threads
  const Geom& G = a.G;
  const int cb = blockIdx.x * 32 + lane;
  const int cbc = cb < G.Vh ? cb : G.Vh - 1;   // lanes past the end work on a valid site
  const int xh = cbc % G.Lxh;
  const int row = cbc / G.Lxh;
  const int y = row % G.Ly;
  const int zt = row / G.Ly;
  const int z = zt % G.Lz;
  const int t = zt / G.Lz;
  const int x = 2 * xh + ((y + z + t + a.out_par) & 1);
  pdl_wait();
  for (int h = w; h < 8; h += RT) {
    const int mu = h >> 1;
    const bool bwd = h & 1;
    int cbf, cbb;
    dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
    const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    const float sg = ((ephase & 1) ? -1.f : 1.f) * (bwd ? -1.f : 1.f);
    float u[18];
    L::load(a.gauge + (size_t)(2 * mu + (bwd ? 1 - a.out_par : a.out_par)) * a.blk_bytes, G.S, bwd ? cbb : cbc, u);
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
  const int rhs0 = (blockIdx.y * RT + w) * NRT;
  if (rhs0 >= a.nrhs) return;
  float acc[NRT][6];
  if constexpr (NRT == 1) {
    // all eight neighbour loads in flight at once
    const size_t rbase = (size_t)rhs0 * a.rhs_stride;
    float v[8][6];
#pragma unroll
    for (int h = 0; h < 8; ++h) VT::load(a.in, rbase + sN[h][lane], v[h]);
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
    static_assert(NRT % 2 == 0, "NRT must be 1 or even");
    // right-hand sides in pairs (lane x: rhs0 + 2p, lane y: rhs0 + 2p + 1); the next hop's
    // vectors are loaded before this hop's arithmetic.  A partial tile repeats the last
    // right-hand side in its loads; the epilogue stores only the valid ones.
    size_t roff[NRT];
#pragma unroll
    for (int r = 0; r < NRT; ++r) roff[r] = (size_t)min(rhs0 + r, a.nrhs - 1) * a.rhs_stride;
    float2 acc2[NRT / 2][6];
#pragma unroll
    for (int p = 0; p < NRT / 2; ++p)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc2[p][k] = make_float2(0.f, 0.f);
    float v[2][NRT][6];
#pragma unroll
    for (int r = 0; r < NRT; ++r) VT::load(a.in, roff[r] + sN[0][lane], v[0][r]);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int cur = h & 1;
      if (h + 1 < 8) {
#pragma unroll
        for (int r = 0; r < NRT; ++r) VT::load(a.in, roff[r] + sN[h + 1][lane], v[cur ^ 1][r]);
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
  pdl_trigger();
  if (cb < G.Vh) {
    double part[NRT];
#pragma unroll
    for (int r = 0; r < NRT; ++r) part[r] = 0.0;
    dslash_epilogue<LQ_F32, NRT, 1>(acc, a.out, a.w1, a.a1, a.w2, a.a2, a.c, RED_NONE, a.rhs_stride, a.nrhs, rhs0,
                                    cb, 0, part);
  }
}

// Shapes of k_dslash_rw: block = 32 x RT threads, rhs_tile = RT x NRT right-hand sides.
inline bool dslash_rw_shape_ok(int block, int tile) {
  if (block % 32 || tile % (block / 32)) return false;
  const int rt = block / 32, nrt = tile / rt;
  return (rt == 2 || rt == 4 || rt == 8) && (nrt == 1 || nrt == 2 || nrt == 4) && rt * nrt <= 16;
}

template <lq_prec GP, int R>
static cudaError_t launch_dslash_rw(const DslashKArgs& k, int block, int tile, cudaStream_t s) {
  if (!dslash_rw_shape_ok(block, tile)) return cudaErrorInvalidValue;
  const int rt = block / 32, nrt = tile / rt;
  dim3 grid((unsigned)((k.G.Vh + 31) / 32), (unsigned)((k.nrhs + tile - 1) / tile));
  const bool pdl = k.pdl != 0;
  switch (rt * 8 + nrt) {
    case 2 * 8 + 1: return launch_k(k_dslash_rw<GP, R, 2, 1>, grid, dim3(64), 0, s, pdl, k);
    case 2 * 8 + 2: return launch_k(k_dslash_rw<GP, R, 2, 2>, grid, dim3(64), 0, s, pdl, k);
    case 2 * 8 + 4: return launch_k(k_dslash_rw<GP, R, 2, 4>, grid, dim3(64), 0, s, pdl, k);
    case 4 * 8 + 1: return launch_k(k_dslash_rw<GP, R, 4, 1>, grid, dim3(128), 0, s, pdl, k);
    case 4 * 8 + 2: return launch_k(k_dslash_rw<GP, R, 4, 2>, grid, dim3(128), 0, s, pdl, k);
    case 4 * 8 + 4: return launch_k(k_dslash_rw<GP, R, 4, 4>, grid, dim3(128), 0, s, pdl, k);
    case 8 * 8 + 1: return launch_k(k_dslash_rw<GP, R, 8, 1>, grid, dim3(256), 0, s, pdl, k);
    case 8 * 8 + 2: return launch_k(k_dslash_rw<GP, R, 8, 2>, grid, dim3(256), 0, s, pdl, k);
    default: return cudaErrorInvalidValue;
  }
}

// Host side: launch one instance.  Supported (rhs tile, threads per site) pairs:
// (1|2, 1|2|4), (4, 1|2), (8, 1), and (RT x NRT, kTpsRhsWarps) for k_dslash_rw;
// dslash_shape_ok() (and dslash_rw_shape_ok()) tell the tuner.
inline bool dslash_shape_ok(int tile, int tps) {
  if (tps == kTpsRhsWarps) return tile >= 2 && tile <= 16;   // with the block: dslash_rw_shape_ok
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
  if (tps == kTpsRhsWarps) {
    if constexpr (GP != LQ_F64 && VP == LQ_F32) {
      if (k.reduce != RED_NONE) return cudaErrorInvalidValue;
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

// Defined in the per-precision translation units.
DslashLaunchFn dslash_fn_f64(int recon);
DslashLaunchFn dslash_fn_f32(int recon);
DslashLaunchFn dslash_fn_bf16(int recon);
DslashLaunchFn dslash_fn_f16(int recon);
