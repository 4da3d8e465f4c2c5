// FP32 multi-RHS hops in packed pairs (included by dslash_site.cuh, which defines
// dslash_neighbours): pairs of right-hand sides share one __ffma2_rn per link element.
#pragma once

#include "lqcd_internal.cuh"

__device__ __forceinline__ void dslash_neighbours(const Geom& G, int mu, int x, int y, int z, int t, int xh,
                                                  int row, int& cbf, int& cbb);

// acc[p] += s * op(U) (v[2p], v[2p+1]) in FP32 with packed FMAs (__ffma2_rn): lane x of
// acc[p][k] is right-hand side 2p, lane y right-hand side 2p+1, and each element of the
// link (times the sign s) is applied to both with one instruction where the scalar form
// needs two.  op(U)_ij is U_ij (ADJ 0) or conj(U_ji) (ADJ 1, Eqs. (1.1)-(2.3)).
template <int ADJ, int NR>
__device__ __forceinline__ void hop_pairs(const float* u, float s, const float (&v)[NR][6],
                                          float2 (&acc)[NR / 2][6]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float er = s * (ADJ ? u[6 * j + 2 * i] : u[6 * i + 2 * j]);
      const float ei = s * (ADJ ? -u[6 * j + 2 * i + 1] : u[6 * i + 2 * j + 1]);
      const float2 E = make_float2(er, er), F = make_float2(ei, ei), N = make_float2(-ei, -ei);
#pragma unroll
      for (int p = 0; p < NR / 2; ++p) {
        const float2 vr = make_float2(v[2 * p][2 * j], v[2 * p + 1][2 * j]);
        const float2 vi = make_float2(v[2 * p][2 * j + 1], v[2 * p + 1][2 * j + 1]);
        acc[p][2 * i] = __ffma2_rn(E, vr, acc[p][2 * i]);
        acc[p][2 * i] = __ffma2_rn(N, vi, acc[p][2 * i]);
        acc[p][2 * i + 1] = __ffma2_rn(E, vi, acc[p][2 * i + 1]);
        acc[p][2 * i + 1] = __ffma2_rn(F, vr, acc[p][2 * i + 1]);
      }
    }
}

// FP32 hops with an even rhs tile: right-hand sides in pairs (hop_pairs), and the next
// hop's link and vectors are loaded before this hop's arithmetic (two buffers), so that a
// thread keeps two hops of loads in flight.  A partial last tile loads the last
// right-hand side again (valid memory, no predicates); the epilogue stores only the valid
// ones.  Hop h = 2j is the forward, h = 2j+1 the backward hop of the thread's direction j.
template <lq_prec GP, int R, lq_prec VP, int NR, int TPS>
__device__ __forceinline__ void dslash_hops_pairs(const char* __restrict__ gauge, size_t blk_bytes, const Geom& G,
                                                  int out_par, const void* __restrict__ in, size_t rhs_stride,
                                                  int nrhs, int rhs0, int cb, int sub, int x, int y, int z, int t,
                                                  int xh, int row, float (&acc)[NR][6]) {
  using L = LinkT<GP, R>;
  using VT = VecT<VP>;
  constexpr int DPT = 4 / TPS;
  constexpr int NH = 2 * DPT;
  const char* hblk[NH];
  int hlink[NH], hnb[NH];
  float hsign[NH];
#pragma unroll
  for (int j = 0; j < DPT; ++j) {
    const int mu = sub * DPT + j;
    int cbf, cbb;
    dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
    const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    const float eta = (ephase & 1) ? -1.f : 1.f;
    hblk[2 * j] = gauge + (size_t)(2 * mu + out_par) * blk_bytes;       // U_mu(x): block (mu, out_par)
    hlink[2 * j] = cb;
    hnb[2 * j] = cbf;
    hsign[2 * j] = eta;
    hblk[2 * j + 1] = gauge + (size_t)(2 * mu + 1 - out_par) * blk_bytes;   // U_mu(x-mu)
    hlink[2 * j + 1] = cbb;
    hnb[2 * j + 1] = cbb;
    hsign[2 * j + 1] = -eta;
  }
  size_t roff[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) roff[r] = (size_t)min(rhs0 + r, nrhs - 1) * rhs_stride;
  float2 acc2[NR / 2][6];
#pragma unroll
  for (int p = 0; p < NR / 2; ++p)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc2[p][k] = make_float2(0.f, 0.f);
  typename L::Raw raw[2];
  float v[2][NR][6];
  raw[0] = L::load_raw(hblk[0], G.S, hlink[0]);
#pragma unroll
  for (int r = 0; r < NR; ++r) VT::load(in, roff[r] + hnb[0], v[0][r]);
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    const int cur = h & 1;
    if (h + 1 < NH) {
      raw[cur ^ 1] = L::load_raw(hblk[h + 1], G.S, hlink[h + 1]);
#pragma unroll
      for (int r = 0; r < NR; ++r) VT::load(in, roff[r] + hnb[h + 1], v[cur ^ 1][r]);
    }
    float u[18];
    L::decode(raw[cur], u);
    if (R == 12) reconstruct_row2(u);
    if (h & 1) hop_pairs<1, NR>(u, hsign[h], v[cur], acc2);
    else hop_pairs<0, NR>(u, hsign[h], v[cur], acc2);
  }
#pragma unroll
  for (int p = 0; p < NR / 2; ++p)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      acc[2 * p][k] += acc2[p][k].x;
      acc[2 * p + 1][k] += acc2[p][k].y;
    }
}

