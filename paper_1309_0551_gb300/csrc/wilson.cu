// Entry point of the Wilson hopping term: dslash_wilson_eo.
#include <stdio.h>

#include <string>
#include <vector>

#include "tune.cuh"
#include "wilson_kernel.cuh"

WilsonLaunchFn wilson_fn_f64(int recon);
WilsonLaunchFn wilson_fn_f32(int recon);
WilsonLaunchFn wilson_fn_16(lq_prec prec, int recon);

namespace {

const char* pname(lq_prec p) { return p == LQ_F64 ? "f64" : p == LQ_F32 ? "f32" : p == LQ_BF16 ? "bf16" : "f16"; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" lq_status dslash_wilson_eo(lq_context* ctx, const lq_gauge* U, const void* in, void* out, int out_parity,
                                      int nrhs, lq_prec vec_prec, int sign, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "gauge is NULL");
  if (!in || !out || !lq_aligned16(in) || !lq_aligned16(out))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out must be non-NULL 16-byte aligned device pointers");
  if (out_parity != 0 && out_parity != 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out_parity must be 0 or 1");
  if (sign != 1 && sign != -1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "sign must be +1 or -1");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  const lq_prec want = U->prec == LQ_F64 ? LQ_F64 : LQ_F32;
  if (vec_prec != want)
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "Wilson spinors must be %s for %s links", pname(want), pname(U->prec));
  const size_t vb = (size_t)nrhs * U->Vh * 24 * lq_prec_bytes(vec_prec);
  if (overlaps(in, vb, out, vb)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in and out overlap");
  DeviceGuard dg(ctx->device);
  WilsonLaunchFn fn = U->prec == LQ_F64 ? wilson_fn_f64(U->recon)
                      : U->prec == LQ_F32 ? wilson_fn_f32(U->recon)
                                          : wilson_fn_16(U->prec, U->recon);
  WilsonKArgs k;
  k.gauge = U->data;
  k.blk_bytes = U->blk_bytes;
  k.G = make_geom(U);
  k.out_par = out_parity;
  k.in = in;
  k.out = out;
  k.rhs_stride = U->Vh;
  cudaStream_t s = (cudaStream_t)stream;
  char key[160];
  snprintf(key, sizeof key, "wilson g=%s/%d dims=%dx%dx%dx%d nrhs=%d", pname(U->prec), (int)U->recon, U->dims[0],
           U->dims[1], U->dims[2], U->dims[3], nrhs);
  TuneEntry pick;
  if (ctx->forced.block) {
    pick = ctx->forced;
  } else {
    std::vector<TuneEntry> cands;
    for (int b : {128, 64, 256}) {
      TuneEntry e;
      e.block = b;
      e.rhs_tile = 1;
      e.tps = 1;
      cands.push_back(e);
    }
    lq_status st = tune_pick(
        ctx, key, cands, s,
        [&](const TuneEntry& c) -> lq_status {
          cudaError_t e = fn(k, sign, c.block, nrhs, s);
          if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_wilson (tuning)");
          return LQ_OK;
        },
        &pick);
    if (st) return st;
  }
  cudaError_t e = fn(k, sign, pick.block, nrhs, s);
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_wilson");
  return LQ_OK;
}
