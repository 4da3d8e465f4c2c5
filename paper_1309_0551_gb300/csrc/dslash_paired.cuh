// Multi-RHS half Dslash on the paired colour-planar vector layout (FP32 vectors).
//
// Layout.  Right-hand sides are taken two at a time.  Pair p of an nrhs-vector field is
// three colour planes of Vh float4 each; element [p][c][site] holds
//   (Re v_2p(site)_c, Re v_2p+1(site)_c, Im v_2p(site)_c, Im v_2p+1(site)_c).
// An odd nrhs has a last pair whose second half is padding (zero after lq_vec_pair, never
// read back by lq_vec_unpair).  A warp of 32 consecutive checkerboard sites reads one
// colour plane of one pair as 512 contiguous bytes (one 16-byte load per lane), and the
// two right-hand sides of a pair are already the two lanes of a packed FP32x2 FMA operand:
// the link element, duplicated once per thread, multiplies both with one __ffma2_rn and no
// register shuffling of vector data.  (The canonical [rhs][site][3] layout makes a thread
// assemble such pairs out of two right-hand sides' 24-byte vectors: register moves that
// outnumber the FMAs.)
//
// Thread mapping.  Lane = site (32 consecutive checkerboard sites per warp); warp w of the
// block takes pair group w % groups (NP pairs = 2 NP right-hand sides) of site chunk
// blockIdx.x * chunks_per_block + w / groups, so the warps that share a site's links sit in
// one block and read them through L1.  Per hop a thread loads the link, rebuilds row 2 for
// 12-real storage, folds the hop's sign (eta_mu(x) forward, -eta_mu(x) backward) into the
// duplicated element and applies it to its NP pairs:
//   Re out += E (Re v) + F (-Im v),  Im out += E (Im v) + F (Re v),  E = (s e_r, s e_r),
//   F = (s e_i, s e_i)  (e = U_ij forward, conj(U_ji) backward).
// Epilogue as the canonical kernels: out = a1 w1 + a2 w2 + c D(in) (w1, w2 paired too),
// optionally with per-rhs Re<w1, out> (RED_DOT) or ||out||^2 (RED_NORM) stored as one
// partial per (rhs, block) -- partials[rhs * gridDim.x + blockIdx.x] -- for a later launch
// to sum (FIN_DEFER).
#pragma once

#include "dslash_site.cuh"
#include "tune.cuh"

struct PairedKArgs {
  const char* gauge;
  size_t blk_bytes;
  Geom G;
  int out_par;
  const float4* in;
  float4* out;
  const float4* w1;
  const float4* w2;
  float a1, a2, c;
  int nrhs;
  int npair;        // (nrhs + 1) / 2
  int groups;       // pair groups per site: ceil(npair / NP) (set by the launcher)
  size_t vstride;   // float4 per colour plane (Vh)
  size_t pstride;   // float4 per pair (3 Vh)
  int reduce;
  Reducer red;
  int pdl;          // host side only
};

constexpr int kPairedMaxWarps = 8;   // blocks of at most 256 threads

// Register caps (blocks of 256 resident per SM): 64 per thread for one pair, 80 for two,
// 128 for four.  Left alone, the compiler hoists the loads of all eight hops and takes 128
// registers in every shape.
constexpr int paired_min_blocks(int np) { return np == 1 ? 4 : np == 2 ? 3 : 2; }

template <lq_prec GP, int R, int NP, bool RED>
__global__ void __launch_bounds__(256, paired_min_blocks(NP)) k_dslash_pr(const PairedKArgs a) {
  using L = LinkT<GP, R>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = w % a.groups;
  const int chunk = blockIdx.x * ((blockDim.x >> 5) / a.groups) + w / a.groups;
  const Geom& G = a.G;
  const int cb = chunk * 32 + lane;
  const bool live = cb < G.Vh;
  const int cbc = live ? cb : G.Vh - 1;   // lanes past the end work on a valid site
  int xh, row, x, y, z, t;
  cb_coords(G, cbc, a.out_par, xh, row, x, y, z, t);
  const int p0 = g * NP;
  size_t poff[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) poff[q] = (size_t)min(p0 + q, a.npair - 1) * a.pstride;
  float2 aR[NP][3], aI[NP][3];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i) aR[q][i] = aI[q][i] = make_float2(0.f, 0.f);
  pdl_wait();
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    const int mu = h >> 1;
    const bool bwd = h & 1;
    int cbf, cbb;
    dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
    const int nb = bwd ? cbb : cbf;
    const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    const float sg = ((ephase & 1) ? -1.f : 1.f) * (bwd ? -1.f : 1.f);
    float u[18];
    L::load(a.gauge + (size_t)(2 * mu + (bwd ? 1 - a.out_par : a.out_par)) * a.blk_bytes, G.S, bwd ? cbb : cbc, u);
    if (R == 12) reconstruct_row2(u);
    float4 v[NP][3];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[q][c] = __ldg(a.in + poff[q] + (size_t)c * a.vstride + nb);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float2 vr[NP], vi[NP], vn[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        vr[q] = make_float2(v[q][j].x, v[q][j].y);
        vi[q] = make_float2(v[q][j].z, v[q][j].w);
        vn[q] = make_float2(-v[q][j].z, -v[q][j].w);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float er = bwd ? u[6 * j + 2 * i] : u[6 * i + 2 * j];
        const float ei = bwd ? -u[6 * j + 2 * i + 1] : u[6 * i + 2 * j + 1];
        const float se = sg * er, sf = sg * ei;
        const float2 E = make_float2(se, se), F = make_float2(sf, sf);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          aR[q][i] = __ffma2_rn(E, vr[q], aR[q][i]);
          aR[q][i] = __ffma2_rn(F, vn[q], aR[q][i]);
          aI[q][i] = __ffma2_rn(E, vi[q], aI[q][i]);
          aI[q][i] = __ffma2_rn(F, vr[q], aI[q][i]);
        }
      }
    }
  }
  pdl_trigger();
  float part[2 * NP];   // summed per warp by the compensated FP32 tree (warp_sum)
#pragma unroll
  for (int r = 0; r < 2 * NP; ++r) part[r] = 0.f;
  if (live) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if (p0 + q >= a.npair) continue;
      const size_t base = (size_t)(p0 + q) * a.pstride + cb;
      float pa = 0.f, pb = 0.f;   // this site's share of rhs 2p and 2p+1
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t o = base + (size_t)c * a.vstride;
        float4 r = make_float4(a.c * aR[q][c].x, a.c * aR[q][c].y, a.c * aI[q][c].x, a.c * aI[q][c].y);
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.w1) {
          w = a.w1[o];
          r.x = fmaf(a.a1, w.x, r.x); r.y = fmaf(a.a1, w.y, r.y);
          r.z = fmaf(a.a1, w.z, r.z); r.w = fmaf(a.a1, w.w, r.w);
        }
        if (a.w2) {
          const float4 w2 = a.w2[o];
          r.x = fmaf(a.a2, w2.x, r.x); r.y = fmaf(a.a2, w2.y, r.y);
          r.z = fmaf(a.a2, w2.z, r.z); r.w = fmaf(a.a2, w2.w, r.w);
        }
        a.out[o] = r;
        if constexpr (RED) {
          if (a.reduce == RED_DOT) {
            pa = fmaf(w.x, r.x, fmaf(w.z, r.z, pa));
            pb = fmaf(w.y, r.y, fmaf(w.w, r.w, pb));
          } else {
            pa = fmaf(r.x, r.x, fmaf(r.z, r.z, pa));
            pb = fmaf(r.y, r.y, fmaf(r.w, r.w, pb));
          }
        }
      }
      part[2 * q] = pa;
      part[2 * q + 1] = pb;
    }
  }
  if constexpr (RED) {
    // per rhs: warp sums, then the block's site chunks of each pair group in chunk order
    __shared__ double sRed[kPairedMaxWarps][2 * NP];
#pragma unroll
    for (int r = 0; r < 2 * NP; ++r) {
      const double s = warp_sum(part[r]);
      if (lane == 0) sRed[w][r] = s;
    }
    __syncthreads();
    const int nchunk = (blockDim.x >> 5) / a.groups;
    if ((int)threadIdx.x < a.groups * 2 * NP) {
      const int gg = threadIdx.x / (2 * NP), r = threadIdx.x % (2 * NP);
      double s = 0.0;
      for (int k = 0; k < nchunk; ++k) s += sRed[k * a.groups + gg][r];
      const int rhs = 2 * gg * NP + r;
      if (rhs < a.nrhs) a.red.partials[(size_t)rhs * gridDim.x + blockIdx.x] = s;
    }
  }
}

// Shapes: NP pairs per thread (1, 2, 4), block of `block` threads (64, 128, 256) holding
// whole pair groups of 32-site chunks.
inline int paired_groups(int npair, int np) { return (npair + np - 1) / np; }
inline bool paired_shape_ok(int npair, int block, int np) {
  if (np != 1 && np != 2 && np != 4) return false;
  if (block != 64 && block != 128 && block != 256) return false;
  return block % (32 * paired_groups(npair, np)) == 0;
}
inline int paired_grid(int Vh, int npair, int block, int np) {
  const int cpb = block / 32 / paired_groups(npair, np);
  const int nchunk = (Vh + 31) / 32;
  return (nchunk + cpb - 1) / cpb;
}

template <lq_prec GP, int R, int NP>
static cudaError_t launch_dslash_pr_np(PairedKArgs k, int block, cudaStream_t s) {
  k.groups = paired_groups(k.npair, NP);
  dim3 grid((unsigned)paired_grid(k.G.Vh, k.npair, block, NP));
  if (k.reduce != RED_NONE) return launch_k(k_dslash_pr<GP, R, NP, true>, grid, dim3(block), 0, s, k.pdl != 0, k);
  return launch_k(k_dslash_pr<GP, R, NP, false>, grid, dim3(block), 0, s, k.pdl != 0, k);
}

template <lq_prec GP, int R>
cudaError_t dslash_paired_launch(const PairedKArgs& k, int block, int np, cudaStream_t s) {
  if (!paired_shape_ok(k.npair, block, np)) return cudaErrorInvalidValue;
  switch (np) {
    case 1: return launch_dslash_pr_np<GP, R, 1>(k, block, s);
    case 2: return launch_dslash_pr_np<GP, R, 2>(k, block, s);
    case 4: return launch_dslash_pr_np<GP, R, 4>(k, block, s);
    default: return cudaErrorInvalidValue;
  }
}

using PairedLaunchFn = cudaError_t (*)(const PairedKArgs&, int block, int np, cudaStream_t);
PairedLaunchFn dslash_paired_fn_f32(int recon);
PairedLaunchFn dslash_paired_fn_bf16(int recon);
PairedLaunchFn dslash_paired_fn_f16(int recon);
