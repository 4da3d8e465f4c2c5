// Per-site pieces of the half staggered Dslash, shared by the single-lattice kernel
// (dslash_kernel.cuh) and the multi-lattice persistent kernel (dslash_multi.cuh).
//
//   out(x) = c * sum_mu eta_mu(x) [ U_mu(x) in(x+mu) - U_mu(x-mu)^dag in(x-mu) ]
//            + a1 * w1(x) + a2 * w2(x)                      (x of parity out_parity)
//
// Forward hops are mult_su3_mat_vec summed over mu (mult_su3_mat_vec_sum_4dir of Table 1);
// backward hops are mult_adj_su3_mat_vec (Eqs. (1.1)-(2.3)), four per site
// (mult_adj_su3_mat_vec_4dir), combined as in sub_four_su3_vecs.  570 flops per site.
//
// TPS threads share one output site (TPS in {1, 2, 4}; consecutive lanes): thread `sub`
// applies the forward and backward hops of directions sub*(4/TPS) ... (sub+1)*(4/TPS)-1,
// the partial sums are combined with xor shuffles, and output colour component c is
// finished and stored by lane c % TPS.  More threads per site put more independent loads
// in flight when the lattice alone would leave the GPU under-occupied.
#pragma once

#include <type_traits>

#include "lqcd_internal.cuh"

// Checkerboard indices of x+mu (cbf) and x-mu (cbb), both on the other parity.
__device__ __forceinline__ void dslash_neighbours(const Geom& G, int mu, int x, int y, int z, int t, int xh,
                                                  int row, int& cbf, int& cbb) {
  if (mu == 0) {
    const int xf = (x + 1 == G.Lx) ? 0 : x + 1;
    const int xb = (x == 0) ? G.Lx - 1 : x - 1;
    cbf = (xf >> 1) + G.Lxh * row;
    cbb = (xb >> 1) + G.Lxh * row;
  } else {
    const int c = (mu == 1) ? y : (mu == 2) ? z : t;
    const int Lm = (mu == 1) ? G.Ly : (mu == 2) ? G.Lz : G.Lt;
    const int sm = (mu == 1) ? 1 : (mu == 2) ? G.Ly : G.Ly * G.Lz;   // row stride
    const int rf = (c + 1 == Lm) ? row - (Lm - 1) * sm : row + sm;
    const int rb = (c == 0) ? row + (Lm - 1) * sm : row - sm;
    cbf = xh + G.Lxh * rf;
    cbb = xh + G.Lxh * rb;
  }
}

#include "dslash_pairs.cuh"

// Accumulates the hops of this thread's directions into acc (zeroed by the caller).  In the
// scalar form, per hop: the link, then the neighbour vectors of every right-hand side, then
// the arithmetic.  (There, issuing both hops' loads first, or the next direction's loads
// before this direction's arithmetic, was measured: the extra registers cost more
// occupancy than they gained.)
template <lq_prec GP, int R, lq_prec VP, int NR, int TPS, class T>
__device__ __forceinline__ void dslash_hops(const char* __restrict__ gauge, size_t blk_bytes, const Geom& G,
                                            int out_par, const void* __restrict__ in, size_t rhs_stride,
                                            int nrhs, int rhs0, int cb, int sub, T (&acc)[NR][6]) {
  using L = LinkT<GP, R>;
  using VT = VecT<VP>;
  constexpr int DPT = 4 / TPS;   // directions per thread
  int xh, row, x, y, z, t;
  cb_coords(G, cb, out_par, xh, row, x, y, z, t);
  const int opar = 1 - out_par;
  if constexpr (std::is_same<T, float>::value && NR % 2 == 0) {
    dslash_hops_pairs<GP, R, VP, NR, TPS>(gauge, blk_bytes, G, out_par, in, rhs_stride, nrhs, rhs0, cb, sub, x, y,
                                          z, t, xh, row, acc);
  } else if constexpr (std::is_same<T, double>::value) {
    // FP64 runs at the FP64 ALU's rate on GB300, so every FP64 instruction counts.  The
    // hop's sign (eta forward, -eta backward) is put on the neighbour vector by flipping
    // its sign bits -- integer XORs, off the FP64 pipe and exact -- and both hops then
    // accumulate straight into acc: 72 FP64 FMAs per direction and rhs.
    constexpr unsigned long long kSign = 0x8000000000000000ull;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int mu = sub * DPT + j;
      int cbf, cbb;
      dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
      const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
      const unsigned long long sf = (ephase & 1) ? kSign : 0ull;   // eta < 0
      T u[18];
      L::load(gauge + (size_t)(2 * mu + out_par) * blk_bytes, G.S, cb, u);
      if (R == 12) reconstruct_row2(u);
      {
        T v[NR][6];
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (rhs0 + r < nrhs) VT::load(in, (size_t)(rhs0 + r) * rhs_stride + cbf, v[r]);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (rhs0 + r < nrhs) {
#pragma unroll
            for (int k = 0; k < 6; ++k) v[r][k] = __longlong_as_double(__double_as_longlong(v[r][k]) ^ sf);
            mat_vec_add(u, v[r], acc[r]);
          }
        }
      }
      L::load(gauge + (size_t)(2 * mu + opar) * blk_bytes, G.S, cbb, u);
      if (R == 12) reconstruct_row2(u);
      {
        T v[NR][6];
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (rhs0 + r < nrhs) VT::load(in, (size_t)(rhs0 + r) * rhs_stride + cbb, v[r]);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (rhs0 + r < nrhs) {
#pragma unroll
            for (int k = 0; k < 6; ++k)
              v[r][k] = __longlong_as_double(__double_as_longlong(v[r][k]) ^ (sf ^ kSign));
            adj_mat_vec_add(u, v[r], acc[r]);
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int mu = sub * DPT + j;
      int cbf, cbb;
      dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
      const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
      const T eta = (ephase & 1) ? T(-1) : T(1);
      T u[18];
      // forward hop: U_mu(x) in(x+mu); U_mu(x) lives in block (mu, out_par) at cb
      L::load(gauge + (size_t)(2 * mu + out_par) * blk_bytes, G.S, cb, u);
      if (R == 12) reconstruct_row2(u);
      {
        T v[NR][6];
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (rhs0 + r < nrhs) VT::load(in, (size_t)(rhs0 + r) * rhs_stride + cbf, v[r]);
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (rhs0 + r < nrhs) mat_vec_acc(u, v[r], acc[r], eta);
      }
      // backward hop: U_mu(x-mu)^dag in(x-mu); that link lives in block (mu, 1-out_par)
      L::load(gauge + (size_t)(2 * mu + opar) * blk_bytes, G.S, cbb, u);
      if (R == 12) reconstruct_row2(u);
      {
        T v[NR][6];
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (rhs0 + r < nrhs) VT::load(in, (size_t)(rhs0 + r) * rhs_stride + cbb, v[r]);
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (rhs0 + r < nrhs) adj_mat_vec_acc(u, v[r], acc[r], -eta);
      }
    }
  }
}

// Combines the TPS partial sums of a site (every lane of the warp must call it).
template <int NR, int TPS, class T>
__device__ __forceinline__ void dslash_combine(T (&acc)[NR][6]) {
#pragma unroll
  for (int off = 1; off < TPS; off <<= 1)
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[r][k] += __shfl_xor_sync(0xffffffffu, acc[r][k], off);
}

// out = c*acc + a1*w1 + a2*w2 for this lane's colour components; adds this lane's share of
// Re<w1, out> (RED_DOT) or ||out||^2 (RED_NORM) to part[r].
// part: the thread's running reduction per rhs, FP64 or (FP32 kernels) FP32, summed per
// warp afterwards by warp_sum / block_reduce.
template <lq_prec VP, int NR, int TPS, class T, class P>
__device__ __forceinline__ void dslash_epilogue(const T (&acc)[NR][6], void* out, const void* w1, double a1,
                                                const void* w2, double a2, double cc, int reduce,
                                                size_t rhs_stride, int nrhs, int rhs0, int cb, int sub,
                                                P (&part)[NR]) {
  using VT = VecT<VP>;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (rhs0 + r < nrhs) {
      const size_t site = (size_t)(rhs0 + r) * rhs_stride + cb;
      T ps = T(0);  // this thread's share of the site's dot or norm, in the vector precision
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (c % TPS != sub) continue;
        T res[2] = {T(cc) * acc[r][2 * c], T(cc) * acc[r][2 * c + 1]};
        T w[2] = {T(0), T(0)};
        if (w1) {
          VT::load_c(w1, site, c, w);
          res[0] = fma(T(a1), w[0], res[0]);
          res[1] = fma(T(a1), w[1], res[1]);
        }
        if (w2) {
          T v2[2];
          VT::load_c(w2, site, c, v2);
          res[0] = fma(T(a2), v2[0], res[0]);
          res[1] = fma(T(a2), v2[1], res[1]);
        }
        VT::store_c(out, site, c, res);
        if (reduce == RED_DOT)
          ps = fma(w[0], res[0], fma(w[1], res[1], ps));
        else if (reduce == RED_NORM)
          ps = fma(res[0], res[0], fma(res[1], res[1], ps));
      }
      part[r] += (P)ps;
    }
  }
}
