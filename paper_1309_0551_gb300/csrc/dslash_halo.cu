// Half staggered Dslash on one sub-domain of a lattice split in t (domain decomposition):
// the sub-domain is a lattice of its own (local t = global t - t0, t0 even, so parities and
// checkerboard indices are the local ones), except that the t hops leaving it read ghost
// data received from the neighbouring sub-domains:
//   forward hop from the last slice:  the input on the next sub-domain's first slice,
//                                     ghost_fwd[rhs][lex_s >> 1];
//   backward hop from the first slice: the input on the previous sub-domain's last slice,
//                                     ghost_bwd[rhs][lex_s >> 1], through its link U_t, held
//                                     in the gauge's halo blocks (lq_gauge_set_halo);
// lex_s = x + Lx (y + Ly z) within the slice.  A face of Vs/2 sites is the first or last
// Vs/2 entries of the sending sub-domain's own one-parity array (Vs = Lx Ly Lz), so faces
// leave without packing.  Epilogue: out = a1 w1 + c D in.  One thread per output site and
// right-hand side (grid.y); 570 flops per site.
#include "dslash_site.cuh"
#include "lqcd_internal.cuh"
#include "tune.cuh"

namespace {

struct HaloArgs {
  const char* gauge;
  size_t blk_bytes;
  Geom G;
  int out_par;
  const void* in;
  void* out;
  const void* ghost_bwd;
  const void* ghost_fwd;
  int Vsh;              // sites of one parity in one time slice
  const char* halo;     // ghost links: two blocks of halo_S chunks per plane
  size_t halo_blk;
  int halo_S;
  const void* w1;
  double a1, c;
};

template <lq_prec GP, int R, lq_prec VP>
__global__ void __launch_bounds__(128) k_dslash_halo(const HaloArgs a) {
  using L = LinkT<GP, R>;
  using VT = VecT<VP>;
  using T = typename L::real;
  const Geom& G = a.G;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= G.Vh) return;
  const int rhs = blockIdx.y;
  const size_t voff = (size_t)rhs * G.Vh, goff = (size_t)rhs * a.Vsh;
  int xh, row, x, y, z, t;
  cb_coords(G, cb, a.out_par, xh, row, x, y, z, t);
  const int opar = 1 - a.out_par;
  T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    int cbf, cbb;
    dslash_neighbours(G, mu, x, y, z, t, xh, row, cbf, cbb);
    const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    const T eta = (ephase & 1) ? T(-1) : T(1);
    T u[18], v[6];
    L::load(a.gauge + (size_t)(2 * mu + a.out_par) * a.blk_bytes, G.S, cb, u);
    if (R == 12) reconstruct_row2(u);
    if (mu == 3 && t == G.Lt - 1) VT::load(a.ghost_fwd, goff + (cb - (size_t)(G.Lt - 1) * a.Vsh), v);
    else VT::load(a.in, voff + cbf, v);
    mat_vec_acc(u, v, acc, eta);
    if (mu == 3 && t == 0) {
      L::load(a.halo + (size_t)opar * a.halo_blk, a.halo_S, cb, u);
      VT::load(a.ghost_bwd, goff + cb, v);
    } else {
      L::load(a.gauge + (size_t)(2 * mu + opar) * a.blk_bytes, G.S, cbb, u);
      VT::load(a.in, voff + cbb, v);
    }
    if (R == 12) reconstruct_row2(u);
    adj_mat_vec_acc(u, v, acc, -eta);
  }
  T res[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) res[k] = T(a.c) * acc[k];
  if (a.w1) {
    T w[6];
    VT::load(a.w1, voff + cb, w);
#pragma unroll
    for (int k = 0; k < 6; ++k) res[k] = fma(T(a.a1), w[k], res[k]);
  }
  VT::store(a.out, voff + cb, res);
}

template <lq_prec GP, int R, lq_prec VP>
cudaError_t launch_halo(const HaloArgs& a, int nrhs, cudaStream_t s) {
  const dim3 grid((a.G.Vh + 127) / 128, nrhs);
  k_dslash_halo<GP, R, VP><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <lq_prec GP>
cudaError_t launch_halo_recon(const HaloArgs& a, int recon, int nrhs, cudaStream_t s) {
  constexpr lq_prec VP = GP == LQ_F64 ? LQ_F64 : LQ_F32;
  return recon == 12 ? launch_halo<GP, 12, VP>(a, nrhs, s) : launch_halo<GP, 18, VP>(a, nrhs, s);
}

}  // namespace

extern "C" lq_status dslash_eo_halo(lq_context* ctx, const lq_gauge* U, const void* in, const void* ghost_bwd,
                                    const void* ghost_fwd, void* out, int out_parity, int nrhs, lq_prec vec_prec,
                                    double a1, const void* w1, double c, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "gauge is NULL");
  if (!U->halo) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "the gauge has no ghost links: call lq_gauge_set_halo");
  if (!in || !out || !ghost_bwd || !ghost_fwd) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "NULL vector");
  if (!lq_aligned16(in) || !lq_aligned16(out) || !lq_aligned16(ghost_bwd) || !lq_aligned16(ghost_fwd) ||
      (w1 && !lq_aligned16(w1)))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "vectors must be 16-byte aligned");
  if (out_parity != 0 && out_parity != 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out_parity must be 0 or 1");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (vec_prec != (U->prec == LQ_F64 ? LQ_F64 : LQ_F32))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "dslash_eo_halo pairs LQ_F64 links with LQ_F64 vectors and "
                                            "reduced-precision links with LQ_F32 vectors");
  if (in == out || (w1 && w1 == out)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out must differ from in and w1");
  DeviceGuard dg(ctx->device);
  HaloArgs a;
  a.gauge = U->data;
  a.blk_bytes = U->blk_bytes;
  a.G = make_geom(U);
  a.out_par = out_parity;
  a.in = in;
  a.out = out;
  a.ghost_bwd = ghost_bwd;
  a.ghost_fwd = ghost_fwd;
  a.Vsh = U->dims[0] * U->dims[1] * U->dims[2] / 2;
  a.halo = U->halo;
  a.halo_blk = U->halo_blk_bytes;
  a.halo_S = U->halo_S;
  a.w1 = w1;
  a.a1 = w1 ? a1 : 0.0;
  a.c = c;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaErrorInvalidValue;
  switch (U->prec) {
    case LQ_F64: e = launch_halo_recon<LQ_F64>(a, (int)U->recon, nrhs, s); break;
    case LQ_F32: e = launch_halo_recon<LQ_F32>(a, (int)U->recon, nrhs, s); break;
    case LQ_BF16: e = launch_halo_recon<LQ_BF16>(a, (int)U->recon, nrhs, s); break;
    case LQ_F16: e = launch_halo_recon<LQ_F16>(a, (int)U->recon, nrhs, s); break;
  }
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_halo");
  return LQ_OK;
}
