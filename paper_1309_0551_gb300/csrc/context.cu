// Context, error reporting, scratch space, gauge packing and the launch-shape autotuner.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include <string>

#include "lqcd_internal.cuh"
#include "tune.cuh"

// ------------------------------------------------------------------ errors -------------

lq_status lq_fail(lq_context* ctx, lq_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

lq_status lq_cuda_fail(lq_context* ctx, cudaError_t e, const char* where) {
  return lq_fail(ctx, LQ_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" const char* lq_status_string(lq_status s) {
  switch (s) {
    case LQ_OK: return "LQ_OK";
    case LQ_ERR_INVALID_ARG: return "LQ_ERR_INVALID_ARG";
    case LQ_ERR_CUDA: return "LQ_ERR_CUDA";
    case LQ_ERR_NOT_CONVERGED: return "LQ_ERR_NOT_CONVERGED";
    case LQ_ERR_NUMERIC: return "LQ_ERR_NUMERIC";
    case LQ_ERR_TIMEOUT: return "LQ_ERR_TIMEOUT";
    case LQ_ERR_UNSUPPORTED: return "LQ_ERR_UNSUPPORTED";
  }
  return "LQ_STATUS_UNKNOWN";
}

extern "C" const char* lq_last_error(const lq_context* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

// ------------------------------------------------------------------ context ------------

extern "C" lq_status lq_create(lq_context** out, int device) {
  if (!out) return LQ_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return LQ_ERR_CUDA;
  if (device < 0 || device >= n) return LQ_ERR_INVALID_ARG;
  lq_context* ctx = new lq_context();
  ctx->device = device;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) { delete ctx; return LQ_ERR_CUDA; }
  ctx->num_sms = prop.multiProcessorCount;
  ctx->l2_bytes = prop.l2CacheSize;
  if (cudaMalloc(&ctx->dev_status, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(ctx->dev_status, 0, sizeof(unsigned int)) != cudaSuccess) {
    if (ctx->dev_status) cudaFree(ctx->dev_status);
    delete ctx;
    return LQ_ERR_CUDA;
  }
  char tag[320];
  snprintf(tag, sizeof tag, "%s/%d", prop.name, prop.multiProcessorCount);
  for (char* c = tag; *c; ++c)
    if (*c == ' ' || *c == '\t') *c = '_';
  ctx->device_tag = tag;
  const char* env = getenv("LQCD_TUNE");
  ctx->tuning = !(env && env[0] == '0');
  // "block,rhs_tile,threads_per_site", e.g. "128,1,2": every Dslash launch whose right-hand
  // side count admits that tile uses this shape instead of the tuned one.
  const char* shape = getenv("LQCD_DSLASH_SHAPE");
  if (shape) {
    int b = 0, t = 0, p = 0;
    if (sscanf(shape, "%d,%d,%d", &b, &t, &p) == 3 && b >= 64 && b <= 256 && b % 32 == 0) {
      ctx->forced.block = b;
      ctx->forced.rhs_tile = t;
      ctx->forced.tps = p;
    }
  }
  const char* cache = getenv("LQCD_TUNE_CACHE");
  if (cache && cache[0]) lq_set_tune_cache(ctx, cache);
  *out = ctx;
  return LQ_OK;
}

// Tuning cache file: one entry per line, "<device tag>\t<key>\t<block> <rhs_tile> <tps> <us>".
// Loading keeps the entries of this device (name and SM count) and leaves entries already
// in the table alone; saving rewrites the file (through a temporary file and a rename) with
// this context's entries plus the other devices' lines it found.
static void tune_load(lq_context* ctx, const std::string& path) {
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    char* t1 = strchr(line, '\t');
    if (!t1) continue;
    char* t2 = strchr(t1 + 1, '\t');
    if (!t2) continue;
    *t1 = 0;
    *t2 = 0;
    if (ctx->device_tag != line) continue;
    TuneEntry e;
    if (sscanf(t2 + 1, "%d %d %d %f", &e.block, &e.rhs_tile, &e.tps, &e.us) != 4 || e.block <= 0) continue;
    ctx->tune.emplace(std::string(t1 + 1), e);
  }
  fclose(f);
}

void lq_tune_save(lq_context* ctx) {
  if (ctx->tune_cache.empty()) return;
  std::string others;
  if (FILE* f = fopen(ctx->tune_cache.c_str(), "r")) {
    char line[1024];
    while (fgets(line, sizeof line, f)) {
      const char* t1 = strchr(line, '\t');
      if (t1 && std::string(line, t1 - line) != ctx->device_tag) others += line;
    }
    fclose(f);
  }
  const std::string tmp = ctx->tune_cache + ".tmp" + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fputs(others.c_str(), f);
  for (const auto& kv : ctx->tune)
    fprintf(f, "%s\t%s\t%d %d %d %.3f\n", ctx->device_tag.c_str(), kv.first.c_str(), kv.second.block,
            kv.second.rhs_tile, kv.second.tps, kv.second.us);
  fclose(f);
  rename(tmp.c_str(), ctx->tune_cache.c_str());
}

extern "C" lq_status lq_set_tune_cache(lq_context* ctx, const char* path) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  ctx->tune_cache = path ? path : "";
  if (!ctx->tune_cache.empty()) tune_load(ctx, ctx->tune_cache);
  return LQ_OK;
}

extern "C" lq_status lq_destroy(lq_context* ctx) {
  if (!ctx) return LQ_OK;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->flush) cudaFree(ctx->flush);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    if (ctx->dev_status) cudaFree(ctx->dev_status);
  }
  delete ctx;
  return LQ_OK;
}

extern "C" lq_status lq_sync(lq_context* ctx, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  LQ_CUDA(ctx, cudaStreamSynchronize(s));
  unsigned int flags = 0;
  LQ_CUDA(ctx, cudaMemcpy(&flags, ctx->dev_status, sizeof flags, cudaMemcpyDeviceToHost));
  if (!flags) return LQ_OK;
  LQ_CUDA(ctx, cudaMemset(ctx->dev_status, 0, sizeof(unsigned int)));
  return lq_fail(ctx, LQ_ERR_TIMEOUT,
                 "a bounded device wait gave up (status flags 0x%x%s): the blocks that waited skipped their "
                 "work, so outputs of the calls issued since the last lq_sync may be unwritten",
                 flags, (flags & kDevTmaTimeout) ? ": TMA bulk copy not delivered" : "");
}

extern "C" lq_status lq_inject_status(lq_context* ctx, unsigned int flags, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int cur = 0;
  LQ_CUDA(ctx, cudaStreamSynchronize(s));
  LQ_CUDA(ctx, cudaMemcpy(&cur, ctx->dev_status, sizeof cur, cudaMemcpyDeviceToHost));
  cur |= flags;
  LQ_CUDA(ctx, cudaMemcpy(ctx->dev_status, &cur, sizeof cur, cudaMemcpyHostToDevice));
  return LQ_OK;
}

extern "C" lq_status lq_set_tuning(lq_context* ctx, int mode) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "tuning mode must be 0, 1 or 2");
  ctx->tuning = mode != 0;
  if (mode) ctx->tune_mode = mode;
  return LQ_OK;
}

extern "C" lq_status lq_tune_report(const lq_context* ctx, char* buf, size_t len, size_t* needed) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  std::string s;
  for (const auto& kv : ctx->tune) {
    char line[256];
    snprintf(line, sizeof line, "%s block=%d rhs_tile=%d tps=%d us=%.3f\n", kv.first.c_str(),
             kv.second.block, kv.second.rhs_tile, kv.second.tps, kv.second.us);
    s += line;
  }
  if (needed) *needed = s.size() + 1;
  if (buf && len) {
    size_t n = s.size() < len - 1 ? s.size() : len - 1;
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return LQ_OK;
}

lq_status lq_scratch(lq_context* ctx, size_t bytes, void** out) {
  if (bytes > ctx->scratch_bytes) {
    // Work queued earlier may still use the old buffer.
    LQ_CUDA(ctx, cudaDeviceSynchronize());
    if (ctx->scratch) LQ_CUDA(ctx, cudaFree(ctx->scratch));
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    size_t want = bytes + (bytes >> 3);
    LQ_CUDA(ctx, cudaMalloc(&ctx->scratch, want));
    LQ_CUDA(ctx, cudaMemset(ctx->scratch, 0, want));
    ctx->scratch_bytes = want;
  }
  *out = ctx->scratch;
  return LQ_OK;
}

lq_status lq_check_dims(lq_context* ctx, const int dims[4]) {
  if (!dims) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "dims is NULL");
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2 || dims[i] % 2)
      return lq_fail(ctx, LQ_ERR_INVALID_ARG, "lattice extent %d is %d: extents must be even and >= 2", i, dims[i]);
    V *= dims[i];
  }
  if (V > (1LL << 30)) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "lattice volume %lld too large", V);
  return LQ_OK;
}

// ------------------------------------------------------------------ gauge packing ------

template <lq_prec P, int R>
__global__ void k_gauge_pack(const double* __restrict__ U, char* __restrict__ out, Geom G,
                             size_t blk_bytes, int V) {
  int lex = blockIdx.x * blockDim.x + threadIdx.x;
  int mu = blockIdx.y;
  if (lex >= V) return;
  const double2* src = reinterpret_cast<const double2*>(U) + ((size_t)mu * V + lex) * 9;
  double u[18];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = src[k];
    u[2 * k] = v.x;
    u[2 * k + 1] = v.y;
  }
  int x = lex % G.Lx;
  int rest = lex / G.Lx;
  int y = rest % G.Ly;
  rest /= G.Ly;
  int z = rest % G.Lz;
  int t = rest / G.Lz;
  int par = (x + y + z + t) & 1;
  int cb = lex >> 1;
  LinkT<P, R>::store(out + (size_t)(2 * mu + par) * blk_bytes, G.S, cb, u);
}

template <lq_prec P, int R>
static size_t link_bytes() { return LinkT<P, R>::bytes_per_site; }

static size_t bytes_per_link(lq_prec p, int r) {
  switch (p) {
    case LQ_F64: return r == 18 ? link_bytes<LQ_F64, 18>() : link_bytes<LQ_F64, 12>();
    case LQ_F32: return r == 18 ? link_bytes<LQ_F32, 18>() : link_bytes<LQ_F32, 12>();
    case LQ_BF16: return r == 18 ? link_bytes<LQ_BF16, 18>() : link_bytes<LQ_BF16, 12>();
    case LQ_F16: return r == 18 ? link_bytes<LQ_F16, 18>() : link_bytes<LQ_F16, 12>();
  }
  return 0;
}

static cudaError_t pack_into(lq_gauge* g, const void* U_canon, cudaStream_t s);

extern "C" lq_status lq_gauge_pack(lq_context* ctx, const int dims[4], const void* U_canon,
                                   lq_prec prec, lq_recon recon, lq_gauge** out, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!out) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  lq_status st = lq_check_dims(ctx, dims);
  if (st) return st;
  if (!U_canon || !lq_aligned16(U_canon))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U must be a non-NULL 16-byte aligned device pointer");
  if (prec < LQ_F64 || prec > LQ_F16) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "bad precision %d", (int)prec);
  if (recon != LQ_RECON_18 && recon != LQ_RECON_12)
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "recon must be 18 or 12");
  DeviceGuard dg(ctx->device);
  lq_gauge* g = new lq_gauge();
  for (int i = 0; i < 4; ++i) g->dims[i] = dims[i];
  int V = dims[0] * dims[1] * dims[2] * dims[3];
  g->Vh = V / 2;
  g->S = (g->Vh + 31) / 32 * 32;
  g->prec = prec;
  g->recon = recon;
  g->blk_bytes = (size_t)g->S * bytes_per_link(prec, recon);
  g->blk_bytes = (g->blk_bytes + 255) / 256 * 256;
  g->bytes = 8 * g->blk_bytes;
  cudaError_t e = cudaMalloc(&g->data, g->bytes);
  if (e != cudaSuccess) { delete g; return lq_cuda_fail(ctx, e, "cudaMalloc(gauge)"); }
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(g->data, 0, g->bytes, s);
  if (e != cudaSuccess) { cudaFree(g->data); delete g; return lq_cuda_fail(ctx, e, "cudaMemsetAsync(gauge)"); }
  e = pack_into(g, U_canon, s);
  if (e != cudaSuccess) { cudaFree(g->data); delete g; return lq_cuda_fail(ctx, e, "k_gauge_pack"); }
  *out = g;
  return LQ_OK;
}

extern "C" lq_status lq_gauge_repack(lq_context* ctx, lq_gauge* g, const void* U_canon, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!g) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "gauge is NULL");
  if (!U_canon || !lq_aligned16(U_canon))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U must be a non-NULL 16-byte aligned device pointer");
  DeviceGuard dg(ctx->device);
  cudaError_t e = pack_into(g, U_canon, (cudaStream_t)stream);
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "k_gauge_pack");
  return LQ_OK;
}

// Launches the packing kernel of g's format over the canonical field U (the padding of the
// planes is left as it is).
static cudaError_t pack_into(lq_gauge* g, const void* U_canon, cudaStream_t s) {
  const int V = 2 * g->Vh;
  const lq_prec prec = g->prec;
  const int recon = (int)g->recon;
  Geom G = make_geom(g);
  dim3 block(256), grid((V + 255) / 256, 4);
#define LQ_PACK(P, R) k_gauge_pack<P, R><<<grid, block, 0, s>>>((const double*)U_canon, g->data, G, g->blk_bytes, V)
  if (recon == 18) {
    switch (prec) {
      case LQ_F64: LQ_PACK(LQ_F64, 18); break;
      case LQ_F32: LQ_PACK(LQ_F32, 18); break;
      case LQ_BF16: LQ_PACK(LQ_BF16, 18); break;
      case LQ_F16: LQ_PACK(LQ_F16, 18); break;
    }
  } else {
    switch (prec) {
      case LQ_F64: LQ_PACK(LQ_F64, 12); break;
      case LQ_F32: LQ_PACK(LQ_F32, 12); break;
      case LQ_BF16: LQ_PACK(LQ_BF16, 12); break;
      case LQ_F16: LQ_PACK(LQ_F16, 12); break;
    }
  }
#undef LQ_PACK
  return cudaGetLastError();
}

extern "C" lq_status lq_gauge_free(lq_context* ctx, lq_gauge* g) {
  if (!g) return LQ_OK;
  if (!ctx) return LQ_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  // The field may still be read by queued work on any stream.
  cudaDeviceSynchronize();
  cudaError_t e = cudaFree(g->data);
  if (g->halo) cudaFree(g->halo);
  delete g;
  if (e != cudaSuccess) return lq_cuda_fail(ctx, e, "cudaFree(gauge)");
  return LQ_OK;
}

// Ghost links of a t-split sub-domain: canonical complex128 U_t of the previous
// sub-domain's last slice, Vs = Lx Ly Lz links in lex order within the slice, into two
// blocks by the parity of the ghost site (x + y + z + 1: it sits at local t = -1), at
// within-face index lex_s >> 1.
template <lq_prec P, int R>
__global__ void k_halo_pack(const double* __restrict__ Ut, char* __restrict__ out, int Lx, int Ly, int Vs, int S,
                            size_t blk_bytes) {
  const int ls = blockIdx.x * blockDim.x + threadIdx.x;
  if (ls >= Vs) return;
  const int x = ls % Lx, y = (ls / Lx) % Ly, z = ls / (Lx * Ly);
  const int par = (x + y + z + 1) & 1;
  const double2* src = reinterpret_cast<const double2*>(Ut) + (size_t)ls * 9;
  double u[18];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 v = src[k];
    u[2 * k] = v.x;
    u[2 * k + 1] = v.y;
  }
  LinkT<P, R>::store(out + (size_t)par * blk_bytes, S, ls >> 1, u);
}

extern "C" lq_status lq_gauge_set_halo(lq_context* ctx, lq_gauge* g, const void* Ut_ghost, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!g || !Ut_ghost || !lq_aligned16(Ut_ghost))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "gauge and a 16-byte aligned ghost-link pointer are required");
  DeviceGuard dg(ctx->device);
  const int Vs = g->dims[0] * g->dims[1] * g->dims[2];
  const int S = (Vs / 2 + 31) / 32 * 32;
  size_t blk = (size_t)S * bytes_per_link(g->prec, g->recon);
  blk = (blk + 255) / 256 * 256;
  if (!g->halo) {
    LQ_CUDA(ctx, cudaMalloc(&g->halo, 2 * blk));
    g->halo_blk_bytes = blk;
    g->halo_S = S;
  }
  cudaStream_t s = (cudaStream_t)stream;
  LQ_CUDA(ctx, cudaMemsetAsync(g->halo, 0, 2 * blk, s));
  const dim3 grid((Vs + 255) / 256), block(256);
  const double* U = (const double*)Ut_ghost;
  const int Lx = g->dims[0], Ly = g->dims[1];
#define LQ_HPACK(P, R) k_halo_pack<P, R><<<grid, block, 0, s>>>(U, g->halo, Lx, Ly, Vs, S, blk)
  if (g->recon == 18) {
    switch (g->prec) {
      case LQ_F64: LQ_HPACK(LQ_F64, 18); break;
      case LQ_F32: LQ_HPACK(LQ_F32, 18); break;
      case LQ_BF16: LQ_HPACK(LQ_BF16, 18); break;
      case LQ_F16: LQ_HPACK(LQ_F16, 18); break;
    }
  } else {
    switch (g->prec) {
      case LQ_F64: LQ_HPACK(LQ_F64, 12); break;
      case LQ_F32: LQ_HPACK(LQ_F32, 12); break;
      case LQ_BF16: LQ_HPACK(LQ_BF16, 12); break;
      case LQ_F16: LQ_HPACK(LQ_F16, 12); break;
    }
  }
#undef LQ_HPACK
  LQ_CHECK_LAUNCH(ctx, "k_halo_pack");
  return LQ_OK;
}

extern "C" lq_status lq_gauge_info(const lq_gauge* g, int dims[4], lq_prec* prec, lq_recon* recon,
                                   size_t* bytes) {
  if (!g) return LQ_ERR_INVALID_ARG;
  if (dims) for (int i = 0; i < 4; ++i) dims[i] = g->dims[i];
  if (prec) *prec = g->prec;
  if (recon) *recon = g->recon;
  if (bytes) *bytes = g->bytes;
  return LQ_OK;
}
