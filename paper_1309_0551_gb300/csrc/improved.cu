// Improved staggered operator entry points: dslash_eo_improved (fat + Naik links) and
// lq_long_links (Naik links from thin links).
#include <stdio.h>

#include <string>
#include <vector>

#include "dslash_improved.cuh"

ImprovedLaunchFn improved_fn_hi(lq_prec p);
ImprovedLaunchFn improved_fn_lo(lq_prec p);
bool dslash_vec_ok(lq_prec gauge, lq_prec vec);

namespace {

const char* pname(lq_prec p) { return p == LQ_F64 ? "f64" : p == LQ_F32 ? "f32" : p == LQ_BF16 ? "bf16" : "f16"; }

std::vector<TuneEntry> improved_candidates(lq_prec gp, int nrhs) {
  std::vector<TuneEntry> c;
  int first = 1;
  for (int t : {1, 2, 4})
    if (t <= nrhs && t <= (gp == LQ_F64 ? 2 : 4)) first = t;
  TuneEntry d;
  d.block = 128; d.rhs_tile = first; d.tps = 1;
  c.push_back(d);
  for (int t : {1, 2, 4}) {
    if (t > nrhs) continue;
    for (int tps : {1, 2})
      for (int b : {64, 128, 256}) {
        if (b == 128 && t == first && tps == 1) continue;
        TuneEntry e;
        e.block = b; e.rhs_tile = t; e.tps = tps;
        c.push_back(e);
      }
  }
  return c;
}

// L_mu(x) = coeff * U_mu(x) U_mu(x+mu) U_mu(x+2mu), canonical complex128 in and out.
__global__ void k_long_links(const double2* __restrict__ U, double2* __restrict__ L, Geom G, int V, double coeff) {
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (lex >= V) return;
  const int x = lex % G.Lx;
  int rest = lex / G.Lx;
  const int y = rest % G.Ly;
  rest /= G.Ly;
  const int z = rest % G.Lz;
  const int t = rest / G.Lz;
  auto shift = [&](int n) {
    const int xs = (mu == 0) ? (x + n) % G.Lx : x;
    const int ys = (mu == 1) ? (y + n) % G.Ly : y;
    const int zs = (mu == 2) ? (z + n) % G.Lz : z;
    const int ts = (mu == 3) ? (t + n) % G.Lt : t;
    return xs + G.Lx * (ys + G.Ly * (zs + G.Lz * ts));
  };
  double a[18], b[18], c[18];
  auto load = [&](int site, double* m) {
    const double2* p = U + ((size_t)mu * V + site) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) { double2 w = p[k]; m[2 * k] = w.x; m[2 * k + 1] = w.y; }
  };
  auto mul = [](const double* A, const double* B, double* C) {   // C = A B
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          re = fma(A[2 * (3 * i + k)], B[2 * (3 * k + j)], re);
          re = fma(-A[2 * (3 * i + k) + 1], B[2 * (3 * k + j) + 1], re);
          im = fma(A[2 * (3 * i + k)], B[2 * (3 * k + j) + 1], im);
          im = fma(A[2 * (3 * i + k) + 1], B[2 * (3 * k + j)], im);
        }
        C[2 * (3 * i + j)] = re;
        C[2 * (3 * i + j) + 1] = im;
      }
  };
  load(lex, a);
  load(shift(1), b);
  mul(a, b, c);
  load(shift(2), b);
  mul(c, b, a);
  double2* q = L + ((size_t)mu * V + lex) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = make_double2(coeff * a[2 * k], coeff * a[2 * k + 1]);
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" lq_status dslash_eo_improved(lq_context* ctx, const lq_gauge* fat, const lq_gauge* lng, const void* in,
                                        void* out, int out_parity, int nrhs, lq_prec vec_prec, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!fat || !lng) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "fat and long gauges are required");
  if (fat->recon != LQ_RECON_18 || lng->recon != LQ_RECON_18 || fat->prec != lng->prec)
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "fat and long links must both be 18-real and of one precision");
  for (int i = 0; i < 4; ++i)
    if (fat->dims[i] != lng->dims[i]) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "fat and long lattices differ");
  if (!in || !out || !lq_aligned16(in) || !lq_aligned16(out))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out must be non-NULL 16-byte aligned device pointers");
  if (out_parity != 0 && out_parity != 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out_parity must be 0 or 1");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (vec_prec < LQ_F64 || vec_prec > LQ_F16 || !dslash_vec_ok(fat->prec, vec_prec))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "vector precision does not pair with the link precision");
  const size_t vb = (size_t)nrhs * fat->Vh * 6 * lq_prec_bytes(vec_prec);
  if (overlaps(in, vb, out, vb)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in and out overlap");
  DeviceGuard dg(ctx->device);
  ImprovedLaunchFn fn = (fat->prec == LQ_F64 || fat->prec == LQ_F32) ? improved_fn_hi(fat->prec)
                                                                      : improved_fn_lo(fat->prec);
  ImpKArgs k;
  k.fat = fat->data;
  k.lng = lng->data;
  k.blk_bytes = fat->blk_bytes;
  k.G = make_geom(fat);
  k.out_par = out_parity;
  k.in = in;
  k.out = out;
  k.rhs_stride = fat->Vh;
  k.nrhs = nrhs;
  cudaStream_t s = (cudaStream_t)stream;
  char key[160];
  snprintf(key, sizeof key, "dslash_improved g=%s v=%s dims=%dx%dx%dx%d nrhs=%d", pname(fat->prec), pname(vec_prec),
           fat->dims[0], fat->dims[1], fat->dims[2], fat->dims[3], nrhs);
  TuneEntry pick;
  const TuneEntry& f = ctx->forced;
  if (f.block && improved_shape_ok(f.rhs_tile, f.tps) && f.rhs_tile <= nrhs) {
    pick = f;
  } else {
    lq_status st = tune_pick(
        ctx, key, improved_candidates(fat->prec, nrhs), s,
        [&](const TuneEntry& c) -> lq_status {
          cudaError_t e = fn(k, vec_prec, c.block, c.rhs_tile, c.tps, s);
          if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_improved (tuning)");
          return LQ_OK;
        },
        &pick);
    if (st) return st;
  }
  cudaError_t e = fn(k, vec_prec, pick.block, pick.rhs_tile, pick.tps, s);
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_improved");
  return LQ_OK;
}

extern "C" lq_status lq_long_links(lq_context* ctx, const int dims[4], const void* U_canon, double coeff,
                                   void* L_canon, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  lq_status st = lq_check_dims(ctx, dims);
  if (st) return st;
  if (!U_canon || !L_canon || !lq_aligned16(U_canon) || !lq_aligned16(L_canon))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U and L must be non-NULL 16-byte aligned device pointers");
  const int V = dims[0] * dims[1] * dims[2] * dims[3];
  const size_t bytes = (size_t)4 * V * 144;
  if (overlaps(U_canon, bytes, L_canon, bytes)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U and L overlap");
  DeviceGuard dg(ctx->device);
  Geom G;
  G.Lx = dims[0]; G.Ly = dims[1]; G.Lz = dims[2]; G.Lt = dims[3];
  G.Lxh = dims[0] / 2; G.Vh = V / 2; G.S = 0;
  dim3 grid((V + 127) / 128, 4);
  k_long_links<<<grid, 128, 0, (cudaStream_t)stream>>>((const double2*)U_canon, (double2*)L_canon, G, V, coeff);
  LQ_CHECK_LAUNCH(ctx, "k_long_links");
  return LQ_OK;
}
