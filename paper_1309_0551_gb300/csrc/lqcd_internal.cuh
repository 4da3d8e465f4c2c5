// Internal declarations shared by the library's translation units: context and gauge
// objects, storage traits for links and colour vectors, error helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>

#include "lqcd.h"

// ------------------------------------------------------------------ host objects -------

struct TuneEntry {
  int block = 0;      // threads per block
  int rhs_tile = 1;   // right-hand sides per thread (Dslash)
  float us = 0.f;     // best measured time
  int tps = 1;        // threads per output site (Dslash); kTpsRhsWarps: the rhs-per-warp kernel
};

// TuneEntry::tps value that selects the multi-RHS Dslash with one thread per (site, rhs):
// blocks of 32 sites x rhs_tile warps, links shared through shared memory (k_dslash_rw).
constexpr int kTpsRhsWarps = 8;
// TuneEntry::tps value that selects the link-staging kernel k_dslash_tma (one thread per
// site, blocks of whole x-rows, links brought into shared memory by TMA bulk copies).
constexpr int kTpsTma = 16;
// TuneEntry::tps value of the paired-layout multi-RHS Dslash k_dslash_pr (rhs_tile = pairs
// of right-hand sides per thread).
constexpr int kTpsPaired = 32;

// Flags of the context's device status word (lq_context::dev_status), set by kernels
// whose bounded waits gave up; lq_sync reports and clears them.
constexpr unsigned int kDevTmaTimeout = 1u;   // a TMA bulk copy did not arrive in time

struct lq_context {
  int device = 0;
  unsigned int* dev_status = nullptr;  // device word of kDev* flags (zero: no failure)
  int num_sms = 0;
  size_t l2_bytes = 0;
  std::string last_error;
  bool tuning = true;
  int tune_mode = 1;            // 1: shapes for lone launches, 2: for concurrent launches
  std::map<std::string, TuneEntry> tune;
  // scratch: reductions (per-block partials, counters), CG scalars, vectors
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* host_pinned = nullptr;  // small pinned buffer for convergence checks
  size_t host_pinned_bytes = 0;
  void* flush = nullptr;        // buffer larger than L2, written between tuning timings
  size_t flush_bytes = 0;
  TuneEntry forced;             // Dslash launch shape forced by LQCD_DSLASH_SHAPE (block 0: none)
  std::string tune_cache;       // file the tuning table is loaded from and saved to ("" = none)
  std::string device_tag;       // "<device name>/<SM count>": entries of other devices are ignored
  std::mutex mu;
};

// Save the context's tuning table to its cache file (no-op without one).
void lq_tune_save(lq_context* ctx);

struct lq_gauge {
  int dims[4];
  int Vh;             // sites per parity
  int S;              // padded sites per parity (plane length), multiple of 32
  lq_prec prec;
  lq_recon recon;
  size_t blk_bytes;   // bytes of one (direction, parity) block
  size_t bytes;       // 8 blocks
  char* data;
  // t-split domain decomposition (lq_gauge_set_halo): U_t on the last slice of the previous
  // sub-domain, the backward links of this sub-domain's first slice, in this gauge's format:
  // two blocks (parity of the ghost site) of halo_S chunks per plane; NULL when not set.
  char* halo = nullptr;
  size_t halo_blk_bytes = 0;
  int halo_S = 0;
};

// Status helpers ------------------------------------------------------------------------
lq_status lq_fail(lq_context* ctx, lq_status s, const char* fmt, ...);
lq_status lq_cuda_fail(lq_context* ctx, cudaError_t e, const char* where);

#define LQ_CUDA(ctx, call)                                              \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return lq_cuda_fail((ctx), _e, #call);       \
  } while (0)

#define LQ_CHECK_LAUNCH(ctx, what)                                      \
  do {                                                                  \
    cudaError_t _e = cudaGetLastError();                                \
    if (_e != cudaSuccess) return lq_cuda_fail((ctx), _e, (what));      \
  } while (0)

inline bool lq_aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
inline size_t lq_prec_bytes(lq_prec p) { return p == LQ_F64 ? 8 : p == LQ_F32 ? 4 : 2; }

// Scratch space of the context (grown on demand, never shrunk).
lq_status lq_scratch(lq_context* ctx, size_t bytes, void** out);
lq_status lq_check_dims(lq_context* ctx, const int dims[4]);

// ------------------------------------------------------------------ device helpers -----

template <class T> struct Cplx { T re, im; };

// A plain load (generic address: global or shared memory), where __ldg needs global.
template <class T> __device__ __forceinline__ T ld_plain(const T* p) { return *p; }

// Link storage: the 18 (or 12) reals of a link, row-major complex (re, im), are split
// into planes; plane k of a (direction, parity) block is an array of S chunks, one chunk
// per site in checkerboard order.  All chunks of a plane have the same width (16, 8 or
// 4 bytes) so a warp reads 32 consecutive chunks: fully coalesced vector loads.
template <lq_prec P, int R> struct LinkT;

// Each format offers load_raw() (the stored chunks, undecoded: issued early, cheap to
// hold), decode() (to reals) and load() = decode(load_raw()); load_raw_plain() reads the
// same plane layout through a generic pointer (a block's copy in shared memory).
template <int R> struct LinkT<LQ_F64, R> {
  using real = double;
  static constexpr int NREAL = R;
  static constexpr size_t bytes_per_site = R * 8;
  struct Raw { double2 c[R / 2]; };
  __device__ __forceinline__ static Raw load_raw(const char* blk, int S, int cb) {
    Raw w;
    const double2* p = reinterpret_cast<const double2*>(blk);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) w.c[k] = __ldg(p + (size_t)k * S + cb);
    return w;
  }
  __device__ __forceinline__ static Raw load_raw_plain(const char* blk, int S, int cb) {
    Raw w;
    const double2* p = reinterpret_cast<const double2*>(blk);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) w.c[k] = ld_plain(p + (size_t)k * S + cb);
    return w;
  }
  __device__ __forceinline__ static void decode(const Raw& w, double* u) {
#pragma unroll
    for (int k = 0; k < R / 2; ++k) { u[2 * k] = w.c[k].x; u[2 * k + 1] = w.c[k].y; }
  }
  __device__ __forceinline__ static void load(const char* blk, int S, int cb, double* u) {
    decode(load_raw(blk, S, cb), u);
  }
  __device__ __forceinline__ static void store(char* blk, int S, int cb, const double* u) {
    double2* p = reinterpret_cast<double2*>(blk);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) p[(size_t)k * S + cb] = make_double2(u[2 * k], u[2 * k + 1]);
  }
};

template <> struct LinkT<LQ_F32, 18> {
  using real = float;
  static constexpr int NREAL = 18;
  static constexpr size_t bytes_per_site = 72;
  struct Raw { float4 a[4]; float2 b; };
  __device__ __forceinline__ static Raw load_raw(const char* blk, int S, int cb) {
    Raw w;
    const float4* p4 = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int k = 0; k < 4; ++k) w.a[k] = __ldg(p4 + (size_t)k * S + cb);
    w.b = __ldg(reinterpret_cast<const float2*>(blk + (size_t)S * 64) + cb);
    return w;
  }
  __device__ __forceinline__ static Raw load_raw_plain(const char* blk, int S, int cb) {
    Raw w;
    const float4* p4 = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int k = 0; k < 4; ++k) w.a[k] = ld_plain(p4 + (size_t)k * S + cb);
    w.b = ld_plain(reinterpret_cast<const float2*>(blk + (size_t)S * 64) + cb);
    return w;
  }
  __device__ __forceinline__ static void decode(const Raw& w, float* u) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u[4 * k] = w.a[k].x; u[4 * k + 1] = w.a[k].y; u[4 * k + 2] = w.a[k].z; u[4 * k + 3] = w.a[k].w;
    }
    u[16] = w.b.x; u[17] = w.b.y;
  }
  __device__ __forceinline__ static void load(const char* blk, int S, int cb, float* u) {
    decode(load_raw(blk, S, cb), u);
  }
  __device__ __forceinline__ static void store(char* blk, int S, int cb, const double* u) {
    float4* p4 = reinterpret_cast<float4*>(blk);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      p4[(size_t)k * S + cb] = make_float4(__double2float_rn(u[4 * k]), __double2float_rn(u[4 * k + 1]),
                                           __double2float_rn(u[4 * k + 2]), __double2float_rn(u[4 * k + 3]));
    float2* p2 = reinterpret_cast<float2*>(blk + (size_t)S * 64);
    p2[cb] = make_float2(__double2float_rn(u[16]), __double2float_rn(u[17]));
  }
};

template <> struct LinkT<LQ_F32, 12> {
  using real = float;
  static constexpr int NREAL = 12;
  static constexpr size_t bytes_per_site = 48;
  struct Raw { float4 a[3]; };
  __device__ __forceinline__ static Raw load_raw(const char* blk, int S, int cb) {
    Raw w;
    const float4* p4 = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int k = 0; k < 3; ++k) w.a[k] = __ldg(p4 + (size_t)k * S + cb);
    return w;
  }
  __device__ __forceinline__ static Raw load_raw_plain(const char* blk, int S, int cb) {
    Raw w;
    const float4* p4 = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int k = 0; k < 3; ++k) w.a[k] = ld_plain(p4 + (size_t)k * S + cb);
    return w;
  }
  __device__ __forceinline__ static void decode(const Raw& w, float* u) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      u[4 * k] = w.a[k].x; u[4 * k + 1] = w.a[k].y; u[4 * k + 2] = w.a[k].z; u[4 * k + 3] = w.a[k].w;
    }
  }
  __device__ __forceinline__ static void load(const char* blk, int S, int cb, float* u) {
    decode(load_raw(blk, S, cb), u);
  }
  __device__ __forceinline__ static void store(char* blk, int S, int cb, const double* u) {
    float4* p4 = reinterpret_cast<float4*>(blk);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      p4[(size_t)k * S + cb] = make_float4(__double2float_rn(u[4 * k]), __double2float_rn(u[4 * k + 1]),
                                           __double2float_rn(u[4 * k + 2]), __double2float_rn(u[4 * k + 3]));
  }
};

// 16-bit storage (bf16 or fp16): conversion helpers.
template <lq_prec P> struct Half16;
template <> struct Half16<LQ_BF16> {
  using h2 = __nv_bfloat162;
  __device__ __forceinline__ static float2 to_f2(uint32_t w) {
    h2 v = *reinterpret_cast<h2*>(&w);
    return __bfloat1622float2(v);
  }
  __device__ __forceinline__ static uint32_t from_d2(double a, double b) {
    __nv_bfloat16 x = __double2bfloat16(a), y = __double2bfloat16(b);
    return (uint32_t)(*reinterpret_cast<uint16_t*>(&x)) | ((uint32_t)(*reinterpret_cast<uint16_t*>(&y)) << 16);
  }
  __device__ __forceinline__ static uint32_t from_f2(float a, float b) {
    h2 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
};
template <> struct Half16<LQ_F16> {
  using h2 = __half2;
  __device__ __forceinline__ static float2 to_f2(uint32_t w) {
    h2 v = *reinterpret_cast<h2*>(&w);
    return __half22float2(v);
  }
  __device__ __forceinline__ static uint32_t from_d2(double a, double b) {
    __half x = __double2half(a), y = __double2half(b);
    return (uint32_t)(*reinterpret_cast<uint16_t*>(&x)) | ((uint32_t)(*reinterpret_cast<uint16_t*>(&y)) << 16);
  }
  __device__ __forceinline__ static uint32_t from_f2(float a, float b) {
    h2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
};

// 16-bit links, 18 reals: two planes of uint4 (8 reals each) + one plane of uint32 (2 reals).
template <lq_prec P, int R> struct Link16;
template <lq_prec P> struct Link16<P, 18> {
  using real = float;
  static constexpr int NREAL = 18;
  static constexpr size_t bytes_per_site = 36;
  struct Raw { uint4 a[2]; uint32_t b; };
  __device__ __forceinline__ static Raw load_raw(const char* blk, int S, int cb) {
    Raw w;
    const uint4* p = reinterpret_cast<const uint4*>(blk);
#pragma unroll
    for (int k = 0; k < 2; ++k) w.a[k] = __ldg(p + (size_t)k * S + cb);
    w.b = __ldg(reinterpret_cast<const uint32_t*>(blk + (size_t)S * 32) + cb);
    return w;
  }
  __device__ __forceinline__ static Raw load_raw_plain(const char* blk, int S, int cb) {
    Raw w;
    const uint4* p = reinterpret_cast<const uint4*>(blk);
#pragma unroll
    for (int k = 0; k < 2; ++k) w.a[k] = ld_plain(p + (size_t)k * S + cb);
    w.b = ld_plain(reinterpret_cast<const uint32_t*>(blk + (size_t)S * 32) + cb);
    return w;
  }
  __device__ __forceinline__ static void decode(const Raw& w, float* u) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float2 a = Half16<P>::to_f2(w.a[k].x), b = Half16<P>::to_f2(w.a[k].y);
      float2 c = Half16<P>::to_f2(w.a[k].z), d = Half16<P>::to_f2(w.a[k].w);
      u[8 * k + 0] = a.x; u[8 * k + 1] = a.y; u[8 * k + 2] = b.x; u[8 * k + 3] = b.y;
      u[8 * k + 4] = c.x; u[8 * k + 5] = c.y; u[8 * k + 6] = d.x; u[8 * k + 7] = d.y;
    }
    float2 e = Half16<P>::to_f2(w.b);
    u[16] = e.x; u[17] = e.y;
  }
  __device__ __forceinline__ static void load(const char* blk, int S, int cb, float* u) {
    decode(load_raw(blk, S, cb), u);
  }
  __device__ __forceinline__ static void store(char* blk, int S, int cb, const double* u) {
    uint4* p = reinterpret_cast<uint4*>(blk);
#pragma unroll
    for (int k = 0; k < 2; ++k)
      p[(size_t)k * S + cb] = make_uint4(Half16<P>::from_d2(u[8 * k], u[8 * k + 1]),
                                         Half16<P>::from_d2(u[8 * k + 2], u[8 * k + 3]),
                                         Half16<P>::from_d2(u[8 * k + 4], u[8 * k + 5]),
                                         Half16<P>::from_d2(u[8 * k + 6], u[8 * k + 7]));
    uint32_t* q = reinterpret_cast<uint32_t*>(blk + (size_t)S * 32);
    q[cb] = Half16<P>::from_d2(u[16], u[17]);
  }
};
// 16-bit links, 12 reals: one plane of uint4 (8 reals) + one plane of uint2 (4 reals).
template <lq_prec P> struct Link16<P, 12> {
  using real = float;
  static constexpr int NREAL = 12;
  static constexpr size_t bytes_per_site = 24;
  struct Raw { uint4 a; uint2 b; };
  __device__ __forceinline__ static Raw load_raw(const char* blk, int S, int cb) {
    Raw w;
    w.a = __ldg(reinterpret_cast<const uint4*>(blk) + cb);
    w.b = __ldg(reinterpret_cast<const uint2*>(blk + (size_t)S * 16) + cb);
    return w;
  }
  __device__ __forceinline__ static Raw load_raw_plain(const char* blk, int S, int cb) {
    Raw w;
    w.a = ld_plain(reinterpret_cast<const uint4*>(blk) + cb);
    w.b = ld_plain(reinterpret_cast<const uint2*>(blk + (size_t)S * 16) + cb);
    return w;
  }
  __device__ __forceinline__ static void decode(const Raw& w, float* u) {
    float2 a = Half16<P>::to_f2(w.a.x), b = Half16<P>::to_f2(w.a.y);
    float2 c = Half16<P>::to_f2(w.a.z), d = Half16<P>::to_f2(w.a.w);
    u[0] = a.x; u[1] = a.y; u[2] = b.x; u[3] = b.y; u[4] = c.x; u[5] = c.y; u[6] = d.x; u[7] = d.y;
    float2 e = Half16<P>::to_f2(w.b.x), f = Half16<P>::to_f2(w.b.y);
    u[8] = e.x; u[9] = e.y; u[10] = f.x; u[11] = f.y;
  }
  __device__ __forceinline__ static void load(const char* blk, int S, int cb, float* u) {
    decode(load_raw(blk, S, cb), u);
  }
  __device__ __forceinline__ static void store(char* blk, int S, int cb, const double* u) {
    uint4* p = reinterpret_cast<uint4*>(blk);
    p[cb] = make_uint4(Half16<P>::from_d2(u[0], u[1]), Half16<P>::from_d2(u[2], u[3]),
                       Half16<P>::from_d2(u[4], u[5]), Half16<P>::from_d2(u[6], u[7]));
    uint2* q = reinterpret_cast<uint2*>(blk + (size_t)S * 16);
    q[cb] = make_uint2(Half16<P>::from_d2(u[8], u[9]), Half16<P>::from_d2(u[10], u[11]));
  }
};
template <int R> struct LinkT<LQ_BF16, R> : Link16<LQ_BF16, R> {};
template <int R> struct LinkT<LQ_F16, R> : Link16<LQ_F16, R> {};

// Colour vectors, canonical layout [rhs][site][3] complex: one chunk per colour.  load()
// goes through the read-only data path and is for data no thread of the kernel writes;
// load_rw() is for arrays the kernel also writes.
template <lq_prec P> struct VecT;
template <> struct VecT<LQ_F64> {
  using real = double;
  static constexpr size_t bytes_per_site = 48;
  __device__ __forceinline__ static void load_c(const void* base, size_t site, int c, double* v) {
    double2 w = __ldg(reinterpret_cast<const double2*>(base) + 3 * site + c);
    v[0] = w.x; v[1] = w.y;
  }
  __device__ __forceinline__ static void store_c(void* base, size_t site, int c, const double* v) {
    reinterpret_cast<double2*>(base)[3 * site + c] = make_double2(v[0], v[1]);
  }
  __device__ __forceinline__ static void load(const void* base, size_t site, double* v) {
    const double2* p = reinterpret_cast<const double2*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) { double2 w = __ldg(p + c); v[2 * c] = w.x; v[2 * c + 1] = w.y; }
  }
  __device__ __forceinline__ static void load_rw(const void* base, size_t site, double* v) {
    const double2* p = reinterpret_cast<const double2*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) { double2 w = p[c]; v[2 * c] = w.x; v[2 * c + 1] = w.y; }
  }
  __device__ __forceinline__ static void store(void* base, size_t site, const double* v) {
    double2* p = reinterpret_cast<double2*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = make_double2(v[2 * c], v[2 * c + 1]);
  }
};
template <> struct VecT<LQ_F32> {
  using real = float;
  static constexpr size_t bytes_per_site = 24;
  __device__ __forceinline__ static void load_c(const void* base, size_t site, int c, float* v) {
    float2 w = __ldg(reinterpret_cast<const float2*>(base) + 3 * site + c);
    v[0] = w.x; v[1] = w.y;
  }
  __device__ __forceinline__ static void store_c(void* base, size_t site, int c, const float* v) {
    reinterpret_cast<float2*>(base)[3 * site + c] = make_float2(v[0], v[1]);
  }
  __device__ __forceinline__ static void load(const void* base, size_t site, float* v) {
    const float2* p = reinterpret_cast<const float2*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) { float2 w = __ldg(p + c); v[2 * c] = w.x; v[2 * c + 1] = w.y; }
  }
  __device__ __forceinline__ static void load_rw(const void* base, size_t site, float* v) {
    const float2* p = reinterpret_cast<const float2*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) { float2 w = p[c]; v[2 * c] = w.x; v[2 * c + 1] = w.y; }
  }
  __device__ __forceinline__ static void store(void* base, size_t site, const float* v) {
    float2* p = reinterpret_cast<float2*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = make_float2(v[2 * c], v[2 * c + 1]);
  }
};
template <lq_prec P> struct Vec16 {
  using real = float;
  static constexpr size_t bytes_per_site = 12;
  __device__ __forceinline__ static void load_c(const void* base, size_t site, int c, float* v) {
    float2 w = Half16<P>::to_f2(__ldg(reinterpret_cast<const uint32_t*>(base) + 3 * site + c));
    v[0] = w.x; v[1] = w.y;
  }
  __device__ __forceinline__ static void store_c(void* base, size_t site, int c, const float* v) {
    reinterpret_cast<uint32_t*>(base)[3 * site + c] = Half16<P>::from_f2(v[0], v[1]);
  }
  __device__ __forceinline__ static void load(const void* base, size_t site, float* v) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) { float2 w = Half16<P>::to_f2(__ldg(p + c)); v[2 * c] = w.x; v[2 * c + 1] = w.y; }
  }
  __device__ __forceinline__ static void load_rw(const void* base, size_t site, float* v) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) { float2 w = Half16<P>::to_f2(p[c]); v[2 * c] = w.x; v[2 * c + 1] = w.y; }
  }
  __device__ __forceinline__ static void store(void* base, size_t site, const float* v) {
    uint32_t* p = reinterpret_cast<uint32_t*>(base) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = Half16<P>::from_f2(v[2 * c], v[2 * c + 1]);
  }
};
template <> struct VecT<LQ_BF16> : Vec16<LQ_BF16> {};
template <> struct VecT<LQ_F16> : Vec16<LQ_F16> {};

// SU(3) arithmetic on interleaved reals (u[2*(3*row+col)+{0,1}], v[2*c+{0,1}]). -----------

// Row 2 of an SU(3) link from rows 0 and 1: conj(row0 x row1).
template <class T> __device__ __forceinline__ void reconstruct_row2(T* u) {
  const T* a = u;       // row 0
  const T* b = u + 6;   // row 1
  // (a x b)_0 = a1 b2 - a2 b1, etc.; the conjugate flips the sign of the imaginary part.
#define LQ_CROSS(i, j, k)                                                                \
  u[12 + 2 * (i)] = (a[2 * (j)] * b[2 * (k)] - a[2 * (j) + 1] * b[2 * (k) + 1]) -       \
                    (a[2 * (k)] * b[2 * (j)] - a[2 * (k) + 1] * b[2 * (j) + 1]);         \
  u[12 + 2 * (i) + 1] = -((a[2 * (j)] * b[2 * (k) + 1] + a[2 * (j) + 1] * b[2 * (k)]) -  \
                          (a[2 * (k)] * b[2 * (j) + 1] + a[2 * (k) + 1] * b[2 * (j)]));
  LQ_CROSS(0, 1, 2)
  LQ_CROSS(1, 2, 0)
  LQ_CROSS(2, 0, 1)
#undef LQ_CROSS
}

// acc += s * U v   (s = +-1 folded in by the caller through sign of v copies)
template <class T> __device__ __forceinline__ void mat_vec_acc(const T* u, const T* v, T* acc, T s) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T re = 0, im = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      re = fma(u[6 * i + 2 * j], v[2 * j], re);
      re = fma(-u[6 * i + 2 * j + 1], v[2 * j + 1], re);
      im = fma(u[6 * i + 2 * j], v[2 * j + 1], im);
      im = fma(u[6 * i + 2 * j + 1], v[2 * j], im);
    }
    acc[2 * i] = fma(s, re, acc[2 * i]);
    acc[2 * i + 1] = fma(s, im, acc[2 * i + 1]);
  }
}

// acc += U v, accumulated in place (no scaling).
template <class T> __device__ __forceinline__ void mat_vec_add(const T* u, const T* v, T* acc) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      acc[2 * i] = fma(u[6 * i + 2 * j], v[2 * j], acc[2 * i]);
      acc[2 * i] = fma(-u[6 * i + 2 * j + 1], v[2 * j + 1], acc[2 * i]);
      acc[2 * i + 1] = fma(u[6 * i + 2 * j], v[2 * j + 1], acc[2 * i + 1]);
      acc[2 * i + 1] = fma(u[6 * i + 2 * j + 1], v[2 * j], acc[2 * i + 1]);
    }
  }
}

// acc += U^dag v, accumulated in place (no scaling).
template <class T> __device__ __forceinline__ void adj_mat_vec_add(const T* u, const T* v, T* acc) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[2 * i] = fma(u[6 * k + 2 * i], v[2 * k], acc[2 * i]);
      acc[2 * i] = fma(u[6 * k + 2 * i + 1], v[2 * k + 1], acc[2 * i]);
      acc[2 * i + 1] = fma(u[6 * k + 2 * i], v[2 * k + 1], acc[2 * i + 1]);
      acc[2 * i + 1] = fma(-u[6 * k + 2 * i + 1], v[2 * k], acc[2 * i + 1]);
    }
  }
}

// acc += s * U^dag v :  (U^dag v)_i = sum_k conj(U_ki) v_k
template <class T> __device__ __forceinline__ void adj_mat_vec_acc(const T* u, const T* v, T* acc, T s) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      re = fma(u[6 * k + 2 * i], v[2 * k], re);
      re = fma(u[6 * k + 2 * i + 1], v[2 * k + 1], re);
      im = fma(u[6 * k + 2 * i], v[2 * k + 1], im);
      im = fma(-u[6 * k + 2 * i + 1], v[2 * k], im);
    }
    acc[2 * i] = fma(s, re, acc[2 * i]);
    acc[2 * i + 1] = fma(s, im, acc[2 * i + 1]);
  }
}

// Programmatic dependent launch.  A kernel launched with the programmatic-serialization
// attribute may be scheduled while its predecessor on the stream drains: it calls
// pdl_wait() before touching anything an earlier kernel writes or reads, and pdl_trigger()
// once its own main work is done (triggering at the start would let the successor's
// blocks occupy SMs that this kernel's remaining blocks still need).  Both are no-ops for
// kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches `kernel` on `s`, with the programmatic-serialization attribute when `pdl`.
template <class... KArgs, class... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Lattice geometry passed to kernels.
// Division by an invariant divisor d >= 1 as a multiply-high, an add and two shifts, exact
// for every 32-bit dividend (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994, in the add-and-shift form that needs no 33-bit multiplier):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, t = hi32(m n) and
// n / d = (t + ((n - t) >> s1)) >> s2, s1 = min(l, 1), s2 = max(l - 1, 0).  The kernels'
// site coordinates need three divisions per thread; as hardware-emulated division by a
// run-time value they cost some 25 instructions each.
struct FastDiv {
  uint32_t m, s1, s2;
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

struct Geom {
  int Lx, Ly, Lz, Lt;
  int Lxh;   // Lx / 2
  int Vh;    // sites per parity
  int S;     // plane length (padded Vh)
  FastDiv dLxh, dLy, dLz;
};

inline Geom make_geom(const lq_gauge* g) {
  Geom G;
  G.Lx = g->dims[0]; G.Ly = g->dims[1]; G.Lz = g->dims[2]; G.Lt = g->dims[3];
  G.Lxh = G.Lx / 2; G.Vh = g->Vh; G.S = g->S;
  G.dLxh = make_fastdiv(G.Lxh);
  G.dLy = make_fastdiv(G.Ly);
  G.dLz = make_fastdiv(G.Lz);
  return G;
}

// Coordinates of the site with checkerboard index cb on parity `par`:
// cb = xh + Lxh * row, row = y + Ly * (z + Lz * t), x = 2 xh + ((y + z + t + par) & 1).
__device__ __forceinline__ void cb_coords(const Geom& G, int cb, int par, int& xh, int& row, int& x, int& y,
                                          int& z, int& t) {
  row = (int)G.dLxh.div((uint32_t)cb);
  xh = cb - row * G.Lxh;
  const int zt = (int)G.dLy.div((uint32_t)row);
  y = row - zt * G.Ly;
  t = (int)G.dLz.div((uint32_t)zt);
  z = zt - t * G.Lz;
  x = 2 * xh + ((y + z + t + par) & 1);
}

// ------------------------------------------------------------------- internal API ------

// Epilogue of the half Dslash used by the solvers:
//   out = a1*w1 + a2*w2 + c*D(in), optional reduction per rhs of Re<w1,out> (RED_DOT)
//   or ||out||^2 (RED_NORM) written to partials[rhs][block] and finished by the last block.
enum { RED_NONE = 0, RED_DOT = 1, RED_NORM = 2 };

struct DslashArgs {
  const lq_gauge* U;
  const void* in;
  void* out;
  int out_parity;
  int nrhs;
  lq_prec vec_prec;
  size_t rhs_stride;   // sites between right-hand sides (normally Vh)
  // epilogue (all optional)
  const void* w1 = nullptr; double a1 = 0.0;
  const void* w2 = nullptr; double a2 = 0.0;
  double c = 1.0;
  int reduce = RED_NONE;
  struct Reducer* red = nullptr;
  bool pdl = false;    // launch with programmatic dependent launch (solver loops)
};

// Deterministic per-rhs reduction: blocks store partials, the last block to finish sums
// them in block order and hands the totals to a finisher.
struct Reducer {
  double* partials;        // [nrhs][nblocks_max]
  unsigned int* counter;   // zero between uses (the last block resets it)
  double* result;          // [nrhs] totals
  int nblocks_max;
  int finisher;            // what the last block does with the totals (solver specific)
  void* finisher_state;    // e.g. CG scalars
  int cols = 0;            // host side: partial columns (row stride) of the last FIN_DEFER launch
};

lq_status launch_dslash(lq_context* ctx, const DslashArgs& a, cudaStream_t s);
