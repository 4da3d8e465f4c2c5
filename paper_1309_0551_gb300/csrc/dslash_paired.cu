// The paired colour-planar FP32 vector layout: conversion to and from the canonical layout
// (lq_vec_pair, lq_vec_unpair) and the multi-RHS half Dslash on it (dslash_eo_paired).
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "dslash_paired.cuh"

// canonical float2 [nrhs][Vh][3] -> paired float4 [npair][3][Vh]; one thread per
// (pair, colour, site); the padding half of an odd last pair is written as zero
__global__ void k_vec_pair(const float2* __restrict__ in, float4* __restrict__ out, int Vh, int nrhs, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int site = (int)(i % Vh);
  const long long pc = i / Vh;
  const int c = (int)(pc % 3), p = (int)(pc / 3);
  const float2 a = in[((size_t)(2 * p) * Vh + site) * 3 + c];
  const float2 b = 2 * p + 1 < nrhs ? in[((size_t)(2 * p + 1) * Vh + site) * 3 + c] : make_float2(0.f, 0.f);
  out[i] = make_float4(a.x, b.x, a.y, b.y);
}

// paired -> canonical; one thread per (rhs, site, colour) of the canonical field
__global__ void k_vec_unpair(const float4* __restrict__ in, float2* __restrict__ out, int Vh, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % 3);
  const long long rs = i / 3;
  const int site = (int)(rs % Vh), r = (int)(rs / Vh);
  const float4 w = in[((size_t)(r >> 1) * 3 + c) * Vh + site];
  out[i] = (r & 1) ? make_float2(w.y, w.w) : make_float2(w.x, w.z);
}

static bool overlap_p(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

// to_paired: `in` canonical and `out` paired (lq_vec_pair), else the reverse
static lq_status vec_pair_check(lq_context* ctx, int Vh, int nrhs, const void* in, void* out, bool to_paired) {
  if (Vh < 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "Vh must be positive");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (!in || !out) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out is NULL");
  if (!lq_aligned16(in) || !lq_aligned16(out)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out must be 16-byte aligned");
  const size_t cb = (size_t)nrhs * Vh * 24, pb = (size_t)((nrhs + 1) / 2) * 3 * Vh * 16;
  if (overlap_p(in, to_paired ? cb : pb, out, to_paired ? pb : cb))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in and out overlap");
  return LQ_OK;
}

extern "C" lq_status lq_vec_pair(lq_context* ctx, int Vh, int nrhs, const void* in, void* out, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (lq_status st = vec_pair_check(ctx, Vh, nrhs, in, out, true)) return st;
  DeviceGuard dg(ctx->device);
  const long long n = (long long)((nrhs + 1) / 2) * 3 * Vh;
  k_vec_pair<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const float2*)in, (float4*)out, Vh, nrhs, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LQ_OK : lq_cuda_fail(ctx, e, "k_vec_pair");
}

extern "C" lq_status lq_vec_unpair(lq_context* ctx, int Vh, int nrhs, const void* in, void* out, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (lq_status st = vec_pair_check(ctx, Vh, nrhs, in, out, false)) return st;
  DeviceGuard dg(ctx->device);
  const long long n = (long long)nrhs * Vh * 3;
  k_vec_unpair<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const float4*)in, (float2*)out, Vh, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LQ_OK : lq_cuda_fail(ctx, e, "k_vec_unpair");
}

static PairedLaunchFn paired_fn(const lq_gauge* g) {
  switch (g->prec) {
    case LQ_F32: return dslash_paired_fn_f32(g->recon);
    case LQ_BF16: return dslash_paired_fn_bf16(g->recon);
    case LQ_F16: return dslash_paired_fn_f16(g->recon);
    default: return nullptr;
  }
}

static const char* gprec_name(lq_prec p) {
  switch (p) {
    case LQ_F32: return "f32";
    case LQ_BF16: return "bf16";
    case LQ_F16: return "f16";
    default: return "?";
  }
}

// Candidate shapes (block, pairs per thread), default first: two pairs per thread (four
// right-hand sides share each loaded link) in blocks of 128.
static std::vector<TuneEntry> paired_candidates(int npair) {
  std::vector<TuneEntry> c;
  auto add = [&](int block, int np) {
    if (!paired_shape_ok(npair, block, np)) return;
    for (const TuneEntry& e : c)
      if (e.block == block && e.rhs_tile == np) return;
    TuneEntry e;
    e.block = block; e.rhs_tile = np; e.tps = kTpsPaired;
    c.push_back(e);
  };
  add(128, npair >= 2 ? 2 : 1);
  for (int np : {1, 2, 4})
    for (int b : {64, 128, 256}) add(b, np);
  return c;
}

// Columns of partials per rhs that a reduction launch of this shape stores (its blocks).
int dslash_paired_cols(int Vh, int nrhs, const TuneEntry& t) {
  return paired_grid(Vh, (nrhs + 1) / 2, t.block, t.rhs_tile);
}

// Launches the paired half Dslash of `k` (out = a1 w1 + a2 w2 + c D(in), optional deferred
// reduction) with a tuned shape.  `red_cols_max`: the partials' row capacity (0 without
// reduction); *cols_out receives the row stride used.
lq_status launch_dslash_paired(lq_context* ctx, const lq_gauge* U, PairedKArgs k, int red_cols_max, int* cols_out,
                               cudaStream_t s) {
  PairedLaunchFn fn = paired_fn(U);
  if (!fn) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "the paired layout takes f32, bf16 or f16 links");
  PairedKArgs plain = k;
  plain.pdl = 0;
  const bool tune_as_is = k.reduce != RED_NONE && k.red.finisher == FIN_DEFER;
  if (!tune_as_is) {
    plain.reduce = RED_NONE;
    plain.w1 = plain.w2 = nullptr;
    plain.a1 = plain.a2 = 0.f;
    plain.c = 1.f;
  }
  TuneEntry pick;
  const TuneEntry& f = ctx->forced;
  if (f.block && f.tps == kTpsPaired && paired_shape_ok(k.npair, f.block, f.rhs_tile)) {
    pick = f;
  } else {
    char key[200];
    snprintf(key, sizeof key, "dslash_paired g=%s/%d dims=%dx%dx%dx%d nrhs=%d%s", gprec_name(U->prec), (int)U->recon,
             U->dims[0], U->dims[1], U->dims[2], U->dims[3], k.nrhs,
             k.reduce == RED_DOT ? " red=dot" : k.reduce == RED_NORM ? " red=norm" : "");
    std::vector<TuneEntry> cands;
    for (const TuneEntry& c : paired_candidates(k.npair))
      if (k.reduce == RED_NONE || dslash_paired_cols(k.G.Vh, k.nrhs, c) <= red_cols_max) cands.push_back(c);
    if (cands.empty()) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "reduction scratch too small");
    lq_status st = tune_pick(
        ctx, key, cands, s,
        [&](const TuneEntry& c) -> lq_status {
          cudaError_t e = fn(plain, c.block, c.rhs_tile, s);
          if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_pr (tuning)");
          return LQ_OK;
        },
        &pick);
    if (st) return st;
  }
  if (k.reduce != RED_NONE) {
    const int cols = dslash_paired_cols(k.G.Vh, k.nrhs, pick);
    if (cols > red_cols_max) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "reduction scratch too small");
    if (cols_out) *cols_out = cols;
  }
  cudaError_t e = fn(k, pick.block, pick.rhs_tile, s);
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_pr");
  return LQ_OK;
}

PairedKArgs make_paired_kargs(const lq_gauge* U, const void* in, void* out, int out_parity, int nrhs) {
  PairedKArgs k;
  memset(&k, 0, sizeof k);
  k.gauge = U->data;
  k.blk_bytes = U->blk_bytes;
  k.G = make_geom(U);
  k.out_par = out_parity;
  k.in = (const float4*)in;
  k.out = (float4*)out;
  k.c = 1.f;
  k.nrhs = nrhs;
  k.npair = (nrhs + 1) / 2;
  k.vstride = (size_t)U->Vh;
  k.pstride = (size_t)3 * U->Vh;
  k.reduce = RED_NONE;
  return k;
}

extern "C" lq_status dslash_eo_paired(lq_context* ctx, const lq_gauge* U, const void* in, void* out, int out_parity,
                                      int nrhs, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "gauge is NULL");
  if (!in || !out) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out is NULL");
  if (!lq_aligned16(in) || !lq_aligned16(out)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out must be 16-byte aligned");
  if (out_parity != 0 && out_parity != 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out_parity must be 0 or 1");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (U->prec == LQ_F64) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "the paired layout takes f32, bf16 or f16 links");
  const size_t vb = (size_t)((nrhs + 1) / 2) * 3 * U->Vh * 16;
  if (overlap_p(in, vb, out, vb)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in and out overlap");
  DeviceGuard dg(ctx->device);
  PairedKArgs k = make_paired_kargs(U, in, out, out_parity, nrhs);
  k.pdl = 1;
  return launch_dslash_paired(ctx, U, k, 0, nullptr, (cudaStream_t)stream);
}
