// The multi-RHS half Dslash with the right-hand sides spread over warps (k_dslash_rw) and
// its launch shapes.
#pragma once

#include "dslash_args.cuh"
#include "dslash_site.cuh"
#include "tune.cuh"

// Multi-RHS half Dslash with the right-hand sides spread over warps: a block holds 32
// sites (lanes) x RT warps, each thread NRT right-hand sides of one site.  Warp w loads the
// links of hop w (and w + RT, ...) for the block's 32 sites once, rebuilds them, folds in
// the hop's sign and writes op(U) (U_mu(x) forward, U_mu(x-mu)^dag backward) to shared
// memory with the neighbour index; after one barrier every thread applies the eight shared
// links to its right-hand sides.  Link loads and the 12-real reconstruction are done once
// per site and hop, not once per rhs; each link element read from shared memory serves
// NRT right-hand sides (in pairs, with packed FP32x2 FMAs, when NRT is even).
// FP32 vectors and arithmetic.  A fused reduction (RED_DOT / RED_NORM of the epilogue) is
// stored, never finished here: every warp owns its right-hand sides, so it writes its
// warp sum to partials[rhs][blockIdx.x] (gridDim.x columns per rhs) and a later launch
// sums the rows (FIN_DEFER).  RED selects the instance with that reduction: the plain
// operator is compiled without it (as a run-time branch it slowed the plain launches by a
// quarter).
template <lq_prec GP, int R, int RT, int NRT, bool RED>
__global__ void __launch_bounds__(32 * RT) k_dslash_rw(const DslashKArgs a) {
  using L = LinkT<GP, R>;
  using VT = VecT<LQ_F32>;
  __shared__ float2 sU[8][9][32];   // [hop][element 3i+j of op(U), sign folded][site]
  __shared__ int sN[8][32];         // [hop][site]: checkerboard index of the neighbour
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // 1-D block of 32 x RT threads
  const Geom& G = a.G;
  const int cb = blockIdx.x * 32 + lane;
  const int cbc = cb < G.Vh ? cb : G.Vh - 1;   // lanes past the end work on a valid site
  int xh, row, x, y, z, t;
  cb_coords(G, cbc, a.out_par, xh, row, x, y, z, t);
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
  float part[NRT];   // summed per warp by the compensated FP32 tree (warp_sum)
#pragma unroll
  for (int r = 0; r < NRT; ++r) part[r] = 0.f;
  if (cb < G.Vh)
    dslash_epilogue<LQ_F32, NRT, 1>(acc, a.out, a.w1, a.a1, a.w2, a.a2, a.c, RED ? a.reduce : RED_NONE, a.rhs_stride,
                                    a.nrhs, rhs0, cb, 0, part);
  if constexpr (RED) {
#pragma unroll
    for (int r = 0; r < NRT; ++r) {
      const double sum = warp_sum(part[r]);
      if (lane == 0 && rhs0 + r < a.nrhs) a.red.partials[(size_t)(rhs0 + r) * gridDim.x + blockIdx.x] = sum;
    }
  }
}

// Shapes of k_dslash_rw: block = 32 x RT threads, rhs_tile = RT x NRT right-hand sides.
inline bool dslash_rw_shape_ok(int block, int tile) {
  if (block % 32 || tile % (block / 32)) return false;
  const int rt = block / 32, nrt = tile / rt;
  return (rt == 2 || rt == 4 || rt == 8) && (nrt == 1 || nrt == 2 || nrt == 4) && rt * nrt <= 16;
}

template <lq_prec GP, int R, bool RED>
static cudaError_t launch_dslash_rw_red(const DslashKArgs& k, int rt, int nrt, cudaStream_t s) {
  dim3 grid((unsigned)((k.G.Vh + 31) / 32), (unsigned)((k.nrhs + rt * nrt - 1) / (rt * nrt)));
  const bool pdl = k.pdl != 0;
  switch (rt * 8 + nrt) {
    case 2 * 8 + 1: return launch_k(k_dslash_rw<GP, R, 2, 1, RED>, grid, dim3(64), 0, s, pdl, k);
    case 2 * 8 + 2: return launch_k(k_dslash_rw<GP, R, 2, 2, RED>, grid, dim3(64), 0, s, pdl, k);
    case 2 * 8 + 4: return launch_k(k_dslash_rw<GP, R, 2, 4, RED>, grid, dim3(64), 0, s, pdl, k);
    case 4 * 8 + 1: return launch_k(k_dslash_rw<GP, R, 4, 1, RED>, grid, dim3(128), 0, s, pdl, k);
    case 4 * 8 + 2: return launch_k(k_dslash_rw<GP, R, 4, 2, RED>, grid, dim3(128), 0, s, pdl, k);
    case 4 * 8 + 4: return launch_k(k_dslash_rw<GP, R, 4, 4, RED>, grid, dim3(128), 0, s, pdl, k);
    case 8 * 8 + 1: return launch_k(k_dslash_rw<GP, R, 8, 1, RED>, grid, dim3(256), 0, s, pdl, k);
    case 8 * 8 + 2: return launch_k(k_dslash_rw<GP, R, 8, 2, RED>, grid, dim3(256), 0, s, pdl, k);
    default: return cudaErrorInvalidValue;
  }
}

template <lq_prec GP, int R>
static cudaError_t launch_dslash_rw(const DslashKArgs& k, int block, int tile, cudaStream_t s) {
  if (!dslash_rw_shape_ok(block, tile)) return cudaErrorInvalidValue;
  const int rt = block / 32, nrt = tile / rt;
  if (k.reduce != RED_NONE) return launch_dslash_rw_red<GP, R, true>(k, rt, nrt, s);
  return launch_dslash_rw_red<GP, R, false>(k, rt, nrt, s);
}

