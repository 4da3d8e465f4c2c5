// dslash_eo entry point and the internal launcher (tuned launch shape) used by the solvers.
#include <stdio.h>

#include <string>
#include <vector>

#include "dslash_kernel.cuh"
#include "dslash_multi.cuh"

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

static const char* prec_name(lq_prec p) {
  switch (p) {
    case LQ_F64: return "f64";
    case LQ_F32: return "f32";
    case LQ_BF16: return "bf16";
    case LQ_F16: return "f16";
  }
  return "?";
}

static DslashLaunchFn pick_fn(const lq_gauge* g) {
  switch (g->prec) {
    case LQ_F64: return dslash_fn_f64(g->recon);
    case LQ_F32: return dslash_fn_f32(g->recon);
    case LQ_BF16: return dslash_fn_bf16(g->recon);
    case LQ_F16: return dslash_fn_f16(g->recon);
  }
  return nullptr;
}

// Sites per block of the link-staging kernel k_dslash_tma for this gauge (0: not used).
static int tma_block(const lq_gauge* g) {
  const Geom G = make_geom(g);
  switch (g->prec) {
    case LQ_F32: return dslash_tma_fn_f32(g->recon)(G);
    case LQ_BF16: return dslash_tma_fn_bf16(g->recon)(G);
    case LQ_F16: return dslash_tma_fn_f16(g->recon)(G);
    default: return 0;
  }
}

bool dslash_vec_ok(lq_prec gauge, lq_prec vec) {
  if (gauge == LQ_F64) return vec == LQ_F64;
  return vec == LQ_F32 || vec == LQ_BF16 || vec == LQ_F16;
}

static std::string dslash_key(const lq_gauge* g, lq_prec vp, int nrhs) {
  char buf[160];
  snprintf(buf, sizeof buf, "dslash g=%s/%d v=%s dims=%dx%dx%dx%d nrhs=%d", prec_name(g->prec),
           (int)g->recon, prec_name(vp), g->dims[0], g->dims[1], g->dims[2], g->dims[3], nrhs);
  return buf;
}

// Candidate launch shapes (block, rhs tile, threads per site), default first.  FP64
// tiles stop at 4 right-hand sides (FP64 accumulators cost two registers each).
static std::vector<TuneEntry> dslash_candidates(lq_prec gp, int nrhs) {
  std::vector<int> tiles;
  for (int t : {1, 2, 4, 8})
    if (t <= nrhs && !(gp == LQ_F64 && t > 4)) tiles.push_back(t);
  int first_tile = 1;
  for (int t : tiles)
    if (t <= (gp == LQ_F64 ? 2 : 4)) first_tile = t;
  std::vector<TuneEntry> c;
  TuneEntry d;
  d.block = 128; d.rhs_tile = first_tile; d.tps = 1;
  c.push_back(d);
  for (int t : tiles)
    for (int tps : {1, 2, 4})
      for (int b : {64, 128, 256}) {
        if (!dslash_shape_ok(t, tps) || (b == 128 && t == first_tile && tps == 1)) continue;
        TuneEntry e;
        e.block = b; e.rhs_tile = t; e.tps = tps;
        c.push_back(e);
      }
  return c;
}

// Columns of per-block partials a reduction launch of this shape stores per rhs: its site
// blocks (32 sites per block for the rhs-per-warp kernel).
static int dslash_partial_cols(int Vh, const TuneEntry& c) {
  if (c.tps == kTpsRhsWarps) return (Vh + 31) / 32;
  if (c.tps == kTpsTma) return (Vh + c.block - 1) / c.block;
  return (int)(((long long)Vh * c.tps + c.block - 1) / c.block);
}

static DslashKArgs make_kargs(const DslashArgs& a) {
  DslashKArgs k;
  k.gauge = a.U->data;
  k.blk_bytes = a.U->blk_bytes;
  k.G = make_geom(a.U);
  k.out_par = a.out_parity;
  k.in = a.in;
  k.out = a.out;
  k.rhs_stride = a.rhs_stride ? a.rhs_stride : (size_t)a.U->Vh;
  k.nrhs = a.nrhs;
  k.w1 = a.w1; k.a1 = a.a1;
  k.w2 = a.w2; k.a2 = a.a2;
  k.c = a.c;
  k.reduce = a.reduce;
  if (a.red) k.red = *a.red;
  else k.red = Reducer{nullptr, nullptr, nullptr, 0, 0, nullptr};
  k.pdl = a.pdl ? 1 : 0;
  k.status = nullptr;
  return k;
}

lq_status launch_dslash(lq_context* ctx, const DslashArgs& a, cudaStream_t s) {
  DslashLaunchFn fn = pick_fn(a.U);
  if (!fn) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "bad gauge precision");
  DslashKArgs k = make_kargs(a);
  k.status = ctx->dev_status;
  // Tuning launches must be repeatable.  A launch without reduction is tuned on the plain
  // operator; a launch with a reduction is tuned as itself (its cost depends on the number
  // of blocks it reduces over), which is repeatable because the solvers never let out alias
  // w1 or w2 and their reductions only store totals or alpha = rr / total.
  // Tuning bursts keep the launch's programmatic dependent launch: a chain of half Dslash
  // calls overlaps each launch's ramp with its predecessor's tail, and the shape that is
  // fastest that way is not always the fastest in isolation.
  DslashKArgs plain = k;
  // a finisher that is not idempotent (FIN_BETA advances the CG state) is never repeated
  const bool tune_as_is = a.reduce != RED_NONE && a.red && a.red->finisher != FIN_BETA;
  if (!tune_as_is) {
    plain.reduce = RED_NONE;
    plain.w1 = plain.w2 = nullptr;
    plain.a1 = plain.a2 = 0.0;
    plain.c = 1.0;
  }
  TuneEntry pick;
  const TuneEntry& f = ctx->forced;
  // the rhs-per-warp kernel: FP32 vectors, two or more rhs, a fused reduction only as
  // deferred per-block partials (FIN_DEFER)
  const bool defer_ok = a.reduce == RED_NONE || (a.red && a.red->finisher == FIN_DEFER);
  const bool rw_ok = a.vec_prec == LQ_F32 && a.U->prec != LQ_F64 && a.nrhs >= 2 && defer_ok;
  // the link-staging kernel: a geometry of whole x-rows per block (tma_block)
  const int tmaT = defer_ok ? tma_block(a.U) : 0;
  if (f.block && dslash_shape_ok(f.rhs_tile, f.tps) && f.rhs_tile <= a.nrhs &&
      !(a.U->prec == LQ_F64 && f.rhs_tile > 4) && (f.tps != kTpsRhsWarps || (rw_ok && dslash_rw_shape_ok(f.block, f.rhs_tile))) &&
      (f.tps != kTpsTma || tmaT > 0)) {
    pick = f;
    if (f.tps == kTpsTma) pick.block = tmaT;
  } else {
    std::string key = dslash_key(a.U, a.vec_prec, a.nrhs);
    std::vector<TuneEntry> cands = dslash_candidates(a.U->prec, a.nrhs);
    if (rw_ok)
      for (int rt : {2, 4, 8})
        for (int nrt : {1, 2, 4}) {
          const int t = rt * nrt;
          if (t > a.nrhs || !dslash_rw_shape_ok(32 * rt, t)) continue;
          TuneEntry e;
          e.block = 32 * rt; e.rhs_tile = t; e.tps = kTpsRhsWarps;
          cands.push_back(e);
        }
    if (tmaT > 0) {
      TuneEntry e;
      e.block = tmaT; e.rhs_tile = 1; e.tps = kTpsTma;
      cands.push_back(e);
    }
    if (a.reduce != RED_NONE) {
      key += a.reduce == RED_DOT ? " red=dot" : " red=norm";
      std::vector<TuneEntry> fit;  // every candidate must fit the reduction scratch
      for (const TuneEntry& c : cands)
        if (a.red && dslash_partial_cols(k.G.Vh, c) <= a.red->nblocks_max) fit.push_back(c);
      if (fit.empty()) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "reduction scratch too small");
      cands = fit;
    }
    lq_status st = tune_pick(
        ctx, key, cands, s,
        [&](const TuneEntry& c) -> lq_status {
          cudaError_t e = fn(plain, a.vec_prec, c.block, c.rhs_tile, c.tps, s);
          if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash (tuning)");
          return LQ_OK;
        },
        &pick);
    if (st) return st;
  }
  if (a.reduce != RED_NONE) {
    const int nbx = dslash_partial_cols(k.G.Vh, pick);
    if (!a.red || nbx > a.red->nblocks_max)
      return lq_fail(ctx, LQ_ERR_INVALID_ARG, "reduction scratch too small");
    a.red->cols = nbx;  // row stride of the partials, for a FIN_DEFER consumer
  }
  cudaError_t e = fn(k, a.vec_prec, pick.block, pick.rhs_tile, pick.tps, s);
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash");
  return LQ_OK;
}


extern "C" lq_status dslash_eo(lq_context* ctx, const lq_gauge* U, const void* in, void* out,
                               int out_parity, int nrhs, lq_prec vec_prec, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "gauge is NULL");
  if (!in || !out) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out is NULL");
  if (!lq_aligned16(in) || !lq_aligned16(out))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in/out must be 16-byte aligned");
  if (out_parity != 0 && out_parity != 1)
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out_parity must be 0 or 1");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  if (vec_prec < LQ_F64 || vec_prec > LQ_F16 || !dslash_vec_ok(U->prec, vec_prec))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "vector precision %d does not pair with gauge precision %d",
                   (int)vec_prec, (int)U->prec);
  size_t vbytes = (size_t)nrhs * U->Vh * 6 * lq_prec_bytes(vec_prec);
  if (overlap(in, vbytes, out, vbytes)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in and out overlap");
  DeviceGuard dg(ctx->device);
  DslashArgs a;
  a.U = U;
  a.in = in;
  a.out = out;
  a.out_parity = out_parity;
  a.nrhs = nrhs;
  a.vec_prec = vec_prec;
  a.rhs_stride = U->Vh;
  // Programmatic dependent launch: the kernel's blocks may be scheduled while the previous
  // kernel on the stream drains; they wait (griddepcontrol.wait) before touching memory,
  // and a predecessor that never triggers early is simply waited for.  Hides the launch
  // and ramp-up of a chain of half Dslash calls.
  a.pdl = true;
  return launch_dslash(ctx, a, (cudaStream_t)stream);
}

// ------------------------------------------------------------ multi-lattice launcher ---

MultiLaunchFn dslash_multi_fn_f64(int recon);
MultiLaunchFn dslash_multi_fn_f32(int recon);
MultiLaunchFn dslash_multi_fn_bf16(int recon);
MultiLaunchFn dslash_multi_fn_f16(int recon);

MultiLaunchFn dslash_multi_fn(lq_prec prec, int recon) {
  switch (prec) {
    case LQ_F64: return dslash_multi_fn_f64(recon);
    case LQ_F32: return dslash_multi_fn_f32(recon);
    case LQ_BF16: return dslash_multi_fn_bf16(recon);
    case LQ_F16: return dslash_multi_fn_f16(recon);
  }
  return nullptr;
}

static std::vector<TuneEntry> multi_candidates(lq_prec gp, int nrhs) {
  std::vector<TuneEntry> c;
  int first_tile = 1;
  for (int t : {1, 2, 4, 8})
    if (t <= nrhs && t <= (gp == LQ_F64 ? 2 : 8)) first_tile = t;
  TuneEntry d;
  d.block = 128; d.rhs_tile = first_tile; d.tps = 1;
  c.push_back(d);
  for (int t : {1, 2, 4, 8}) {
    if (t > nrhs || (gp == LQ_F64 && t > 4)) continue;
    for (int tps : {1, 2, 4})
      for (int b : {64, 128, 256}) {
        if (!dslash_multi_shape_ok(t, tps) || (b == 128 && t == first_tile && tps == 1)) continue;
        TuneEntry e;
        e.block = b; e.rhs_tile = t; e.tps = tps;
        c.push_back(e);
      }
  }
  return c;
}

// Launches the multi-lattice half Dslash described by `a` (lattice table, vectors,
// epilogue) with a tuned launch shape; `key` names the lattice set for the tuning table.
lq_status launch_dslash_multi(lq_context* ctx, MultiKArgs a, lq_prec gp, int recon, lq_prec vp,
                              const std::string& key, cudaStream_t s) {
  MultiLaunchFn fn = dslash_multi_fn(gp, recon);
  if (!fn) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "bad gauge precision");
  // Tuning launches must be repeatable: the plain operator, or a launch with a reduction
  // tuned as itself (its cost depends on the shape; the solvers never let out alias w1 or
  // w2, and their finishers only store totals or alpha = rr / total).
  MultiKArgs plain = a;
  // a finisher that is not idempotent (FIN_BETA advances the CG state) is never repeated
  const bool tune_as_is = a.reduce != RED_NONE && a.red.finisher != FIN_BETA;
  if (!tune_as_is) {
    for (int l = 0; l < a.nlat; ++l) plain.lat[l].w1 = plain.lat[l].w2 = nullptr;
    plain.c = 1.0;
    plain.skip_state = nullptr;
    plain.reduce = RED_NONE;
  }
  const bool rw_ok = gp != LQ_F64 && vp == LQ_F32 && a.nrhs >= 2;
  TuneEntry pick;
  const TuneEntry& f = ctx->forced;
  if (f.block && dslash_multi_shape_ok(f.rhs_tile, f.tps) && f.rhs_tile <= a.nrhs &&
      !(gp == LQ_F64 && f.rhs_tile > 4) && (f.tps != kTpsRhsWarps || (rw_ok && dslash_rw_shape_ok(f.block, f.rhs_tile)))) {
    pick = f;
  } else {
    std::vector<TuneEntry> cands = multi_candidates(gp, a.nrhs);
    if (rw_ok)
      for (int rt : {2, 4, 8})
        for (int nrt : {1, 2, 4}) {
          const int t = rt * nrt;
          if (t > a.nrhs || !dslash_rw_shape_ok(32 * rt, t)) continue;
          TuneEntry e;
          e.block = 32 * rt; e.rhs_tile = t; e.tps = kTpsRhsWarps;
          cands.push_back(e);
        }
    std::string tkey = key;
    // (a reduction launch stores one partial column per block; its grid is capped at the
    // partials' row stride, so every candidate fits)
    if (a.reduce != RED_NONE) tkey += a.reduce == RED_DOT ? " red=dot" : " red=norm";
    lq_status st = tune_pick(
        ctx, tkey, cands, s,
        [&](const TuneEntry& c) -> lq_status {
          cudaError_t e = fn(plain, vp, c.block, c.rhs_tile, c.tps, ctx->num_sms, s);
          if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_multi (tuning)");
          return LQ_OK;
        },
        &pick);
    if (st) return st;
  }
  if (a.reduce != RED_NONE && a.pstride < 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "reduction scratch too small");
  cudaError_t e = fn(a, vp, pick.block, pick.rhs_tile, pick.tps, ctx->num_sms, s);
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_dslash_multi");
  return LQ_OK;
}

extern "C" lq_status dslash_eo_multi(lq_context* ctx, int nlat, const lq_gauge* const* U, const void* const* in,
                                     void* const* out, int out_parity, int nrhs, lq_prec vec_prec,
                                     lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (nlat < 1 || nlat > kMaxLat) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nlat must be in [1, %d]", kMaxLat);
  if (!U || !in || !out) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "NULL array argument");
  if (out_parity != 0 && out_parity != 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out_parity must be 0 or 1");
  if (nrhs < 1 || nrhs > 16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  for (int l = 0; l < nlat; ++l) {
    if (!U[l]) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U[%d] is NULL", l);
    if (U[l]->prec != U[0]->prec || U[l]->recon != U[0]->recon)
      return lq_fail(ctx, LQ_ERR_INVALID_ARG, "all gauges must share precision and recon");
    if (!in[l] || !out[l] || !lq_aligned16(in[l]) || !lq_aligned16(out[l]))
      return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in[%d]/out[%d] must be non-NULL 16-byte aligned", l, l);
    const size_t vb = (size_t)nrhs * U[l]->Vh * 6 * lq_prec_bytes(vec_prec);
    if (overlap(in[l], vb, out[l], vb)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "in[%d] and out[%d] overlap", l, l);
  }
  const lq_prec gp = U[0]->prec;
  if ((gp == LQ_F64 && vec_prec != LQ_F64) || (gp != LQ_F64 && vec_prec != LQ_F32))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "dslash_eo_multi pairs LQ_F64 links with LQ_F64 vectors and "
                                            "reduced-precision links with LQ_F32 vectors");
  DeviceGuard dg(ctx->device);
  MultiKArgs a;
  memset(&a, 0, sizeof a);
  a.nlat = nlat;
  a.nrhs = nrhs;
  a.out_par = out_parity;
  a.c = 1.0;
  a.reduce = RED_NONE;
  std::string lats;
  for (int l = 0; l < nlat; ++l) {
    a.lat[l].gauge = U[l]->data;
    a.lat[l].blk_bytes = U[l]->blk_bytes;
    a.lat[l].G = make_geom(U[l]);
    a.lat[l].in = in[l];
    a.lat[l].out = out[l];
    char d[64];
    snprintf(d, sizeof d, "%s%dx%dx%dx%d", l ? "," : "", U[l]->dims[0], U[l]->dims[1], U[l]->dims[2], U[l]->dims[3]);
    lats += d;
  }
  char key[512];
  snprintf(key, sizeof key, "dslash_multi g=%s/%d v=%s lats=%s nrhs=%d", prec_name(gp), (int)U[0]->recon,
           prec_name(vec_prec), lats.c_str(), nrhs);
  return launch_dslash_multi(ctx, a, gp, U[0]->recon, vec_prec, key, (cudaStream_t)stream);
}
