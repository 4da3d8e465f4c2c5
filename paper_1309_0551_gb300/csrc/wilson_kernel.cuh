// Wilson hopping term on one parity, through half Wilson vectors:
//
//   out(x) = sum_mu [ (1 - s gamma_mu) U_mu(x) in(x+mu) + (1 + s gamma_mu) U_mu(x-mu)^dag in(x-mu) ]
//
// for x of parity out_par, s = SIGN = +1 or -1 (the adjoint), gamma matrices in the
// DeGrand-Rossi basis.  (1 + e gamma_mu) has rank two: in that basis gamma_mu =
// [[0, B_mu], [B_mu^dag, 0]], so (1 + e gamma_mu) psi = (h, e B_mu^dag h) with
// h = psi_up + e B_mu psi_down.  Each hop therefore projects the neighbour spinor to a half
// Wilson vector h (two colour vectors), multiplies it by the link -- mult_su3_mat_hwvec
// forward, mult_adj_su3_mat_hwvec backward (Table 1) -- and adds (g, e B^dag g) to the
// accumulator.  1320 flops per output site.
//
// The B_mu, with multiplications by +-1 and +-i written out:
//   x: B = [[0, i], [i, 0]]    y: B = [[0, -1], [1, 0]]    z: B = [[i, 0], [0, -i]]    t: B = 1
//
// A spinor is 24 reals [spin][colour][re, im]; fields are [nrhs][Vh][4][3] complex.
#pragma once

#include "lqcd_internal.cuh"

struct WilsonKArgs {
  const char* gauge;
  size_t blk_bytes;
  Geom G;
  int out_par;
  const void* in;
  void* out;
  size_t rhs_stride;
};

// 24-real spinor loads and stores with 16-byte accesses.
template <lq_prec VP> struct SpinorT;
template <> struct SpinorT<LQ_F64> {
  using real = double;
  static constexpr size_t bytes_per_site = 192;
  __device__ __forceinline__ static void load(const void* base, size_t site, double (&p)[24]) {
    const double2* q = reinterpret_cast<const double2*>(base) + 12 * site;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double2 w = __ldg(q + k);
      p[2 * k] = w.x;
      p[2 * k + 1] = w.y;
    }
  }
  __device__ __forceinline__ static void store(void* base, size_t site, const double (&p)[24]) {
    double2* q = reinterpret_cast<double2*>(base) + 12 * site;
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = make_double2(p[2 * k], p[2 * k + 1]);
  }
};
template <> struct SpinorT<LQ_F32> {
  using real = float;
  static constexpr size_t bytes_per_site = 96;
  __device__ __forceinline__ static void load(const void* base, size_t site, float (&p)[24]) {
    const float4* q = reinterpret_cast<const float4*>(base) + 6 * site;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 w = __ldg(q + k);
      p[4 * k] = w.x;
      p[4 * k + 1] = w.y;
      p[4 * k + 2] = w.z;
      p[4 * k + 3] = w.w;
    }
  }
  __device__ __forceinline__ static void store(void* base, size_t site, const float (&p)[24]) {
    float4* q = reinterpret_cast<float4*>(base) + 6 * site;
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = make_float4(p[4 * k], p[4 * k + 1], p[4 * k + 2], p[4 * k + 3]);
  }
};

// Real and imaginary part of spin s, colour c in a spinor / half vector.
#define WRE(v, s, c) v[6 * (s) + 2 * (c)]
#define WIM(v, s, c) v[6 * (s) + 2 * (c) + 1]

// h = psi_up + E * B_MU psi_down (E = +1 or -1).
template <int MU, int E, class T>
__device__ __forceinline__ void half_project(const T (&p)[24], T (&h)[12]) {
  const T e = T(E);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {          // h0 = p0 + e i p3, h1 = p1 + e i p2
      WRE(h, 0, c) = fma(-e, WIM(p, 3, c), WRE(p, 0, c));
      WIM(h, 0, c) = fma(e, WRE(p, 3, c), WIM(p, 0, c));
      WRE(h, 1, c) = fma(-e, WIM(p, 2, c), WRE(p, 1, c));
      WIM(h, 1, c) = fma(e, WRE(p, 2, c), WIM(p, 1, c));
    } else if (MU == 1) {   // h0 = p0 - e p3, h1 = p1 + e p2
      WRE(h, 0, c) = fma(-e, WRE(p, 3, c), WRE(p, 0, c));
      WIM(h, 0, c) = fma(-e, WIM(p, 3, c), WIM(p, 0, c));
      WRE(h, 1, c) = fma(e, WRE(p, 2, c), WRE(p, 1, c));
      WIM(h, 1, c) = fma(e, WIM(p, 2, c), WIM(p, 1, c));
    } else if (MU == 2) {   // h0 = p0 + e i p2, h1 = p1 - e i p3
      WRE(h, 0, c) = fma(-e, WIM(p, 2, c), WRE(p, 0, c));
      WIM(h, 0, c) = fma(e, WRE(p, 2, c), WIM(p, 0, c));
      WRE(h, 1, c) = fma(e, WIM(p, 3, c), WRE(p, 1, c));
      WIM(h, 1, c) = fma(-e, WRE(p, 3, c), WIM(p, 1, c));
    } else {                // h0 = p0 + e p2, h1 = p1 + e p3
      WRE(h, 0, c) = fma(e, WRE(p, 2, c), WRE(p, 0, c));
      WIM(h, 0, c) = fma(e, WIM(p, 2, c), WIM(p, 0, c));
      WRE(h, 1, c) = fma(e, WRE(p, 3, c), WRE(p, 1, c));
      WIM(h, 1, c) = fma(e, WIM(p, 3, c), WIM(p, 1, c));
    }
  }
}

// acc += (g, E * B_MU^dag g) for the transported half vector g.
template <int MU, int E, class T>
__device__ __forceinline__ void half_accumulate(const T (&g)[12], T (&acc)[24]) {
  const T e = T(E);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] += g[k];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {          // B^dag = [[0, -i], [-i, 0]]: lower = (-e i g1, -e i g0)
      WRE(acc, 2, c) = fma(e, WIM(g, 1, c), WRE(acc, 2, c));
      WIM(acc, 2, c) = fma(-e, WRE(g, 1, c), WIM(acc, 2, c));
      WRE(acc, 3, c) = fma(e, WIM(g, 0, c), WRE(acc, 3, c));
      WIM(acc, 3, c) = fma(-e, WRE(g, 0, c), WIM(acc, 3, c));
    } else if (MU == 1) {   // B^dag = [[0, 1], [-1, 0]]: lower = (e g1, -e g0)
      WRE(acc, 2, c) = fma(e, WRE(g, 1, c), WRE(acc, 2, c));
      WIM(acc, 2, c) = fma(e, WIM(g, 1, c), WIM(acc, 2, c));
      WRE(acc, 3, c) = fma(-e, WRE(g, 0, c), WRE(acc, 3, c));
      WIM(acc, 3, c) = fma(-e, WIM(g, 0, c), WIM(acc, 3, c));
    } else if (MU == 2) {   // B^dag = [[-i, 0], [0, i]]: lower = (-e i g0, e i g1)
      WRE(acc, 2, c) = fma(e, WIM(g, 0, c), WRE(acc, 2, c));
      WIM(acc, 2, c) = fma(-e, WRE(g, 0, c), WIM(acc, 2, c));
      WRE(acc, 3, c) = fma(-e, WIM(g, 1, c), WRE(acc, 3, c));
      WIM(acc, 3, c) = fma(e, WRE(g, 1, c), WIM(acc, 3, c));
    } else {                // B^dag = 1: lower = (e g0, e g1)
      WRE(acc, 2, c) = fma(e, WRE(g, 0, c), WRE(acc, 2, c));
      WIM(acc, 2, c) = fma(e, WIM(g, 0, c), WIM(acc, 2, c));
      WRE(acc, 3, c) = fma(e, WRE(g, 1, c), WRE(acc, 3, c));
      WIM(acc, 3, c) = fma(e, WIM(g, 1, c), WIM(acc, 3, c));
    }
  }
}

#undef WRE
#undef WIM

// Both hops of direction MU for the output site at checkerboard index cb; cbf / cbb are
// the checkerboard indices of x+mu and x-mu on the other parity.
template <lq_prec GP, int R, lq_prec VP, int MU, int SIGN, class T>
__device__ __forceinline__ void wilson_direction(const WilsonKArgs& a, size_t rbase, int cb, int cbf, int cbb,
                                                 T (&acc)[24]) {
  using L = LinkT<GP, R>;
  using ST = SpinorT<VP>;
  T u[18], p[24], h[12], g[12];
  // forward: (1 - s gamma_mu) U_mu(x) in(x+mu); U_mu(x) lives in block (mu, out_par)
  L::load(a.gauge + (size_t)(2 * MU + a.out_par) * a.blk_bytes, a.G.S, cb, u);
  if (R == 12) reconstruct_row2(u);
  ST::load(a.in, rbase + cbf, p);
  half_project<MU, -SIGN>(p, h);
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k] = T(0);
  mat_vec_add(u, h, g);
  mat_vec_add(u, h + 6, g + 6);
  half_accumulate<MU, -SIGN>(g, acc);
  // backward: (1 + s gamma_mu) U_mu(x-mu)^dag in(x-mu); that link lives in block (mu, 1-out_par)
  L::load(a.gauge + (size_t)(2 * MU + 1 - a.out_par) * a.blk_bytes, a.G.S, cbb, u);
  if (R == 12) reconstruct_row2(u);
  ST::load(a.in, rbase + cbb, p);
  half_project<MU, SIGN>(p, h);
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k] = T(0);
  adj_mat_vec_add(u, h, g);
  adj_mat_vec_add(u, h + 6, g + 6);
  half_accumulate<MU, SIGN>(g, acc);
}

// One thread per output site; grid = (site blocks, nrhs).
template <lq_prec GP, int R, lq_prec VP, int SIGN>
__global__ void __launch_bounds__(256) k_wilson(const WilsonKArgs a) {
  using T = typename LinkT<GP, R>::real;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= a.G.Vh) return;
  const Geom& G = a.G;
  int xh, row, x, y, z, t;   // row = y + Ly*(z + Lz*t)
  cb_coords(G, cb, a.out_par, xh, row, x, y, z, t);
  const size_t rbase = (size_t)blockIdx.y * a.rhs_stride;
  // neighbours on the other parity
  const int xf = (x + 1 == G.Lx) ? 0 : x + 1;
  const int xb = (x == 0) ? G.Lx - 1 : x - 1;
  const int ryf = (y + 1 == G.Ly) ? row - (G.Ly - 1) : row + 1;
  const int ryb = (y == 0) ? row + (G.Ly - 1) : row - 1;
  const int rzf = (z + 1 == G.Lz) ? row - (G.Lz - 1) * G.Ly : row + G.Ly;
  const int rzb = (z == 0) ? row + (G.Lz - 1) * G.Ly : row - G.Ly;
  const int yz = G.Ly * G.Lz;
  const int rtf = (t + 1 == G.Lt) ? row - (G.Lt - 1) * yz : row + yz;
  const int rtb = (t == 0) ? row + (G.Lt - 1) * yz : row - yz;
  T acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = T(0);
  wilson_direction<GP, R, VP, 0, SIGN>(a, rbase, cb, (xf >> 1) + G.Lxh * row, (xb >> 1) + G.Lxh * row, acc);
  wilson_direction<GP, R, VP, 1, SIGN>(a, rbase, cb, xh + G.Lxh * ryf, xh + G.Lxh * ryb, acc);
  wilson_direction<GP, R, VP, 2, SIGN>(a, rbase, cb, xh + G.Lxh * rzf, xh + G.Lxh * rzb, acc);
  wilson_direction<GP, R, VP, 3, SIGN>(a, rbase, cb, xh + G.Lxh * rtf, xh + G.Lxh * rtb, acc);
  SpinorT<VP>::store(a.out, rbase + cb, acc);
}

using WilsonLaunchFn = cudaError_t (*)(const WilsonKArgs&, int sign, int block, int nrhs, cudaStream_t);

template <lq_prec GP, int R>
cudaError_t wilson_launch(const WilsonKArgs& k, int sign, int block, int nrhs, cudaStream_t s) {
  constexpr lq_prec VP = GP == LQ_F64 ? LQ_F64 : LQ_F32;
  dim3 grid((unsigned)((k.G.Vh + block - 1) / block), (unsigned)nrhs);
  if (sign > 0) k_wilson<GP, R, VP, 1><<<grid, block, 0, s>>>(k);
  else k_wilson<GP, R, VP, -1><<<grid, block, 0, s>>>(k);
  return cudaGetLastError();
}
