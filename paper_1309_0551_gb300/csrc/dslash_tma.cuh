// The half Dslash with every link a block needs staged in shared memory by TMA bulk copies
// (k_dslash_tma).
//
// A block covers T = nr * Lx/2 sites: nr whole x-rows of one xy-plane (row = y + Ly(z + Lz t),
// cb = xh + Lx/2 * row).  Then each of the eight hops needs its links from ONE contiguous
// run of checkerboard indices of its (direction, parity) block, two at the y wrap:
//   forward hops, and the backward x hop:  the block's own range [c0, c0 + T);
//   backward y:  the rows one below, [c0 - Lx/2, ...), or, for a block starting at y = 0,
//                the wrap row y = Ly - 1 of the same plane followed by [c0, c0 + T - Lx/2);
//   backward z:  the plane below (z - 1, or Lz - 1); backward t: the slab below (t - 1, or
//                Lt - 1).
// Placed in shared memory so that every hop but the backward x one reads its link at the
// thread's own index, each run is one cp.async.bulk per storage plane: one warp issues all
// of them at block start, so the block's 8 T links are in flight at once (what a lone
// launch on a small lattice lacks: a few blocks per SM, one load chain per thread), each
// hop on its own mbarrier so that the arithmetic starts when hop 0 has landed.  The
// neighbour vectors (4-8% of the bytes) come through L1/L2 as in k_dslash, issued before
// the waits.  Every wait is bounded (tma.cuh): on expiry the thread records kDevTmaTimeout
// in the status word, waits once more for the remaining hops and stores nothing.
// Measured on GB300 it runs slower than k_dslash in every regime timed (16^3 x 32 and 32^4,
// one launch at a time or four in flight): it holds 12-24 warps per SM where k_dslash
// holds up to 40, and k_dslash's coalesced loads already bring the links at the copy
// bandwidth.  It stays a tuner candidate, picked only where it is the fastest.
// FP32 arithmetic (links of FP32, BF16 or FP16 storage, vectors of the same precisions),
// one thread per site, the block's right-hand sides one after another over the staged
// links; a fused reduction is stored as per-block partials (FIN_DEFER).
#pragma once

#include "dslash_args.cuh"
#include "dslash_site.cuh"
#include "tma.cuh"
#include "tune.cuh"

// Shared memory a block's links may take (so that two blocks fit an SM).
constexpr size_t kTmaMaxSmem = 112 * 1024;

// Storage planes of a link format (the LinkT layouts): count and chunk bytes of plane k.
template <lq_prec P, int R> struct TmaPlanes {
  static constexpr int n = P == LQ_F32 ? (R == 18 ? 5 : 3) : (R == 18 ? 3 : 2);
  __host__ __device__ static constexpr int chunk(int k) {
    return P == LQ_F32 ? (R == 18 && k == 4 ? 8 : 16) : (k == 0 ? 16 : k == 1 ? (R == 18 ? 16 : 8) : 4);
  }
  __host__ __device__ static constexpr int min_chunk() { return P == LQ_F32 ? (R == 18 ? 8 : 16) : (R == 18 ? 4 : 8); }
};

// Sites per block for this geometry and link size, or 0 when the kernel does not apply:
// the largest T = nr * Lx/2 with nr | Ly, T a multiple of 32 in [64, 256], 8 T links within
// kTmaMaxSmem; runs start at multiples of Lx/2, so 8-byte planes need Lx/2 even and
// 4-byte planes Lx/2 a multiple of 4 (16-byte aligned copies).
inline int dslash_tma_sites(const Geom& G, size_t link_bytes, int min_chunk) {
  if ((min_chunk == 8 && G.Lxh % 2) || (min_chunk == 4 && G.Lxh % 4)) return 0;
  int best = 0;
  for (int nr = 1; nr <= G.Ly; ++nr) {
    if (G.Ly % nr) continue;
    const int T = nr * G.Lxh;
    if (T % 32 || T < 64 || T > 256 || 8 * (size_t)T * link_bytes > kTmaMaxSmem) continue;
    best = T;   // the largest: fewer, larger copies (runs of 64 sites, 0.5-1 KB, ran slower)
  }
  return best;
}

// One contiguous run of a hop's links: n links from checkerboard index src of the hop's
// (direction, parity) block to shared-memory index dst.
struct TmaRun { int src, dst, n; };

// The runs of hop h (= 2 mu + backward) for the block starting at c0 with T sites; returns
// their count (1 or 2).
__device__ __forceinline__ int tma_hop_runs(const Geom& G, int h, int c0, int T, TmaRun (&r)[2]) {
  const int mu = h >> 1;
  const bool bwd = h & 1;
  const int row0 = c0 / G.Lxh;   // c0 is a multiple of Lx/2 (uniform: no fast path needed)
  const int Ps = G.Lxh * G.Ly;   // sites of one xy-plane
  if (!bwd || mu == 0) {
    r[0] = {c0, 0, T};
    return 1;
  }
  if (mu == 1) {
    if (row0 % G.Ly) {
      r[0] = {c0 - G.Lxh, 0, T};
      return 1;
    }
    r[0] = {c0 + (G.Ly - 1) * G.Lxh, 0, G.Lxh};   // the wrap row y = Ly - 1
    r[1] = {c0, G.Lxh, T - G.Lxh};
    return 2;
  }
  const int plane = row0 / G.Ly;   // z + Lz t
  if (mu == 2) {
    const int z = plane % G.Lz;
    r[0] = {z ? c0 - Ps : c0 + (G.Lz - 1) * Ps, 0, T};
    return 1;
  }
  const int t = plane / G.Lz;
  r[0] = {t ? c0 - Ps * G.Lz : c0 + (G.Lt - 1) * Ps * G.Lz, 0, T};
  return 1;
}

template <lq_prec GP, int R, lq_prec VP, bool RED>
__global__ void __launch_bounds__(256) k_dslash_tma(const DslashKArgs a, int T) {
  using L = LinkT<GP, R>;
  using VT = VecT<VP>;
  using PL = TmaPlanes<GP, R>;
  constexpr int kLink = (int)L::bytes_per_site;
  extern __shared__ __align__(128) unsigned char sm[];   // [hop][plane][T chunks]
  __shared__ uint64_t bar[8];                              // one per hop: compute starts with hop 0
  const Geom& G = a.G;
  const int c0 = blockIdx.x * T;
  const int i = threadIdx.x;
  const int cb = c0 + i;   // < Vh: T divides Vh
  int xh, row, x, y, z, t;
  cb_coords(G, cb, a.out_par, xh, row, x, y, z, t);
  int nb[8], lidx[8];
  float sg[8];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    int cbf, cbb;
    dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
    const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    const float eta = (ephase & 1) ? -1.f : 1.f;
    nb[2 * mu] = cbf;
    nb[2 * mu + 1] = cbb;
    lidx[2 * mu] = i;
    lidx[2 * mu + 1] = mu == 0 ? cbb - c0 : i;
    sg[2 * mu] = eta;
    sg[2 * mu + 1] = -eta;
  }
  pdl_wait();   // the links and the input may be written by the previous kernel
  if (threadIdx.x < 32) {
    if (threadIdx.x < 8) {
      tma::mbar_init(&bar[threadIdx.x], 1);
      tma::mbar_expect_tx(&bar[threadIdx.x], (uint32_t)(T * kLink));
    }
    __syncwarp();
    // the warp's lanes share out the (hop, run, plane) copies, hop 0 first
    int item = 0;
#pragma unroll 1
    for (int h = 0; h < 8; ++h) {
      TmaRun runs[2];
      const int nr = tma_hop_runs(G, h, c0, T, runs);
      const int mu = h >> 1;
      const char* blk = a.gauge + (size_t)(2 * mu + ((h & 1) ? 1 - a.out_par : a.out_par)) * a.blk_bytes;
      unsigned char* hs = sm + (size_t)h * T * kLink;
      int pre = 0;   // bytes of the planes before plane k, per site
#pragma unroll
      for (int k = 0; k < PL::n; ++k) {
        const int ch = PL::chunk(k);
        for (int q = 0; q < nr; ++q, ++item) {
          if ((item & 31) != (int)threadIdx.x) continue;
          tma::load(hs + (size_t)T * pre + (size_t)runs[q].dst * ch, blk + (size_t)G.S * pre + (size_t)runs[q].src * ch,
                    (uint32_t)(runs[q].n * ch), &bar[h]);
        }
        pre += ch;
      }
    }
  }
  __syncthreads();   // the barriers are initialised before anyone waits on them
  bool ok = true;
  for (int rhs = 0; rhs < a.nrhs; ++rhs) {
    const size_t voff = (size_t)rhs * a.rhs_stride;
    float v[8][6];
#pragma unroll
    for (int h = 0; h < 8; ++h) VT::load(a.in, voff + nb[h], v[h]);   // in flight with the links
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      if (rhs == 0 && ok && !tma::mbar_wait(&bar[h], 0)) {
        ok = false;
        atomicOr(a.status, kDevTmaTimeout);
        for (int g = h; g < 8; ++g) tma::mbar_wait(&bar[g], 0);   // once more, bounded
      }
      float u[18];
      L::decode(L::load_raw_plain(reinterpret_cast<const char*>(sm + (size_t)h * T * kLink), T, lidx[h]), u);
      if (R == 12) reconstruct_row2(u);
      if (h & 1) adj_mat_vec_acc(u, v[h], acc, sg[h]);
      else mat_vec_acc(u, v[h], acc, sg[h]);
    }
    float res[6];
    float part[1] = {0.f};
#pragma unroll
    for (int k = 0; k < 6; ++k) res[k] = (float)a.c * acc[k];
    float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (a.w1) {
      VT::load(a.w1, voff + cb, w);
#pragma unroll
      for (int k = 0; k < 6; ++k) res[k] = fmaf((float)a.a1, w[k], res[k]);
    }
    if (a.w2) {
      float w2v[6];
      VT::load(a.w2, voff + cb, w2v);
#pragma unroll
      for (int k = 0; k < 6; ++k) res[k] = fmaf((float)a.a2, w2v[k], res[k]);
    }
    if (ok) VT::store(a.out, voff + cb, res);   // a block whose links did not arrive writes nothing
    if constexpr (RED) {
      // the site's share in the working precision (six products), summed per warp by the
      // compensated FP32 tree and in FP64 from there
      float ps = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) ps = fmaf(a.reduce == RED_DOT ? w[k] : res[k], res[k], ps);
      part[0] = ok ? ps : 0.f;
      block_sum_store<1>(part, a.red.partials + (size_t)rhs * gridDim.x + blockIdx.x, 1, 1);
    }
  }
  pdl_trigger();
}

// Host: sites per block of the link-staging kernel for a gauge format, 0 if it does not apply.
template <lq_prec GP, int R>
inline int dslash_tma_block(const Geom& G) {
  if constexpr (GP == LQ_F64) {
    return 0;   // FP64 is bound by the FP64 pipe, not by link latency
  } else {
    return dslash_tma_sites(G, LinkT<GP, R>::bytes_per_site, TmaPlanes<GP, R>::min_chunk());
  }
}

template <lq_prec GP, int R, lq_prec VP>
static cudaError_t launch_dslash_tma(const DslashKArgs& k, cudaStream_t s) {
  if constexpr (GP == LQ_F64) {
    return cudaErrorInvalidValue;
  } else {
    const int T = dslash_tma_block<GP, R>(k.G);
    if (!T || k.G.Vh % T || !k.status) return cudaErrorInvalidValue;
    if (k.reduce != RED_NONE && k.red.finisher != FIN_DEFER) return cudaErrorInvalidValue;
    const size_t smem = 8 * (size_t)T * LinkT<GP, R>::bytes_per_site;
    void (*kern)(const DslashKArgs, int) =
        k.reduce != RED_NONE ? k_dslash_tma<GP, R, VP, true> : k_dslash_tma<GP, R, VP, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaMaxSmem);
    if (e != cudaSuccess) return e;
    return launch_k(kern, dim3((unsigned)(k.G.Vh / T)), dim3(T), smem, s, k.pdl != 0, k, T);
  }
}
