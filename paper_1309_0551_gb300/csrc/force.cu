// Fermion force of S = Re chi^dag (m^2 - D_eo D_oe) chi, chi on the even sites.
//
//   psi = D_oe chi                                   (half Dslash, ||psi||^2 fused)
//   dS/dchi = 2 M chi = 2 m^2 chi - 2 D_eo psi        (half Dslash with fused epilogue
//                                                     and Re<chi, 2 M chi> = 2 S)
//   per link U_mu(y):  Z =  eta_mu(y) chi(y+mu) psi(y)^dag      (y odd)
//                      Z = -eta_mu(y) psi(y+mu) chi(y)^dag      (y even)
//   (su3_projector outer products of Table 1), G = dS/dU = 2 Z^dag, F = TA(U G^dag),
//   TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6.
// psi is recomputed from chi on every call rather than kept from a forward pass.
#include <math.h>
#include <string.h>

#include <vector>

#include "lqcd_internal.cuh"
#include "tune.cuh"

namespace {

constexpr int kForceThreads = 128;

// Complex helpers on (re, im) pairs.
template <class T> struct C2 { T r, i; };
template <class T> __device__ __forceinline__ C2<T> cmul_conj(C2<T> a, C2<T> b) {  // a * conj(b)
  return {a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i};
}

// Copies `nreal` reals from shared to global memory with 16-byte stores (both 16-byte
// aligned; the block's slice starts at a multiple of kForceThreads links).
template <class T>
__device__ __forceinline__ void store_slice(T* __restrict__ dst, const T* __restrict__ src, int nreal) {
  constexpr int W = 16 / sizeof(T);
  const int nvec = nreal / W;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x)
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
  for (int i = nvec * W + threadIdx.x; i < nreal; i += blockDim.x) dst[i] = src[i];
}

// One thread per link (mu = blockIdx.y, lex); G and F leave through shared memory so that
// each block writes its contiguous slice of the [4][V][3][3] outputs with coalesced stores.
template <lq_prec P>
__global__ void __launch_bounds__(kForceThreads) k_force(const char* __restrict__ gauge, size_t blk_bytes, Geom G,
                                                         const void* __restrict__ chi, const void* __restrict__ psi,
                                                         void* __restrict__ dSdU, void* __restrict__ fta) {
  using L = LinkT<P, 18>;
  using VT = VecT<P>;
  using T = typename L::real;
  __shared__ __align__(16) T stage[kForceThreads * 18];
  const int V = 2 * G.Vh;
  const int lex0 = blockIdx.x * blockDim.x;
  const int lex = lex0 + threadIdx.x;
  const int mu = blockIdx.y;
  const int nlinks = min((int)blockDim.x, V - lex0);
  const bool live = lex < V;
  T g[18], f[18];
  if (live) {
    const int x = lex % G.Lx;
    int rest = lex / G.Lx;
    const int y = rest % G.Ly;
    rest /= G.Ly;
    const int z = rest % G.Lz;
    const int t = rest / G.Lz;
    const int par = (x + y + z + t) & 1;
    const int cb = lex >> 1;
    // neighbour y + mu (periodic)
    const int xf = (mu == 0) ? (x + 1 == G.Lx ? 0 : x + 1) : x;
    const int yf = (mu == 1) ? (y + 1 == G.Ly ? 0 : y + 1) : y;
    const int zf = (mu == 2) ? (z + 1 == G.Lz ? 0 : z + 1) : z;
    const int tf = (mu == 3) ? (t + 1 == G.Lt ? 0 : t + 1) : t;
    const int lexf = xf + G.Lx * (yf + G.Ly * (zf + G.Lz * tf));
    const int cbf = lexf >> 1;
    const int ephase = (mu == 0) ? 0 : (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    const T eta = (ephase & 1) ? T(-1) : T(1);
    // a = left vector, b = right vector of the outer product Z = s * a b^dag
    T a[6], b[6];
    T s;
    if (par) {  // y odd: chi(y+mu) psi(y)^dag
      VT::load(chi, cbf, a);
      VT::load(psi, cb, b);
      s = eta;
    } else {    // y even: -psi(y+mu) chi(y)^dag
      VT::load(psi, cbf, a);
      VT::load(chi, cb, b);
      s = -eta;
    }
    T u[18];
    L::load(gauge + (size_t)(2 * mu + par) * blk_bytes, G.S, cb, u);
    // With a' = 2 s a:  G = 2 Z^dag = b a'^dag  (G_ij = b_i conj(a'_j)), and
    // A = U G^dag = U a' b^dag = (U a') b^dag:  the link product is a mat-vec followed by
    // an outer product (su3_projector, Table 1), not a 3x3 matrix product.
    T ap[6], w[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      ap[k] = T(2) * s * a[k];
      w[k] = T(0);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const C2<T> q = cmul_conj(C2<T>{b[2 * i], b[2 * i + 1]}, C2<T>{ap[2 * j], ap[2 * j + 1]});
        g[2 * (3 * i + j)] = q.r;
        g[2 * (3 * i + j) + 1] = q.i;
      }
    mat_vec_add(u, ap, w);
    {
      C2<T> A[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = cmul_conj(C2<T>{w[2 * i], w[2 * i + 1]}, C2<T>{b[2 * j], b[2 * j + 1]});
      // TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6 * 1; Tr(A - A^dag) = 2i Im Tr A
      const T trim = (A[0][0].i + A[1][1].i + A[2][2].i) / T(3);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          f[2 * (3 * i + j)] = T(0.5) * (A[i][j].r - A[j][i].r);
          f[2 * (3 * i + j) + 1] = T(0.5) * (A[i][j].i + A[j][i].i) - (i == j ? trim : T(0));
        }
    }
  }  // live
  const size_t slice = ((size_t)mu * V + lex0) * 18;  // first real of this block's links
  if (dSdU) {
    if (live)
#pragma unroll
      for (int k = 0; k < 18; ++k) stage[threadIdx.x * 18 + k] = g[k];
    __syncthreads();
    store_slice(reinterpret_cast<T*>(dSdU) + slice, stage, nlinks * 18);
    __syncthreads();
  }
  if (fta) {
    if (live)
#pragma unroll
      for (int k = 0; k < 18; ++k) stage[threadIdx.x * 18 + k] = f[k];
    __syncthreads();
    store_slice(reinterpret_cast<T*>(fta) + slice, stage, nlinks * 18);
  }
}

}  // namespace

extern "C" lq_status dslash_force(lq_context* ctx, const lq_gauge* U, double mass, const void* chi, void* dSdU,
                                  void* force_TA, void* dSdchi, double* S, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!U || !chi) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "U and chi are required");
  if (U->recon != LQ_RECON_18 || (U->prec != LQ_F64 && U->prec != LQ_F32))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "dslash_force needs an 18-real LQ_F64 or LQ_F32 gauge");
  if (!lq_aligned16(chi) || (dSdU && !lq_aligned16(dSdU)) || (force_TA && !lq_aligned16(force_TA)) ||
      (dSdchi && !lq_aligned16(dSdchi)))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
  DeviceGuard dg(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const lq_prec vp = U->prec;
  const size_t es = lq_prec_bytes(vp);
  const size_t vbytes = (size_t)U->Vh * 6 * es;
  const int nblocks_max = (U->Vh + 15) / 16;
  // scratch: psi, dS/dchi (when the caller passes none), 1 scalar, counter, partials
  const size_t need = 2 * vbytes + 64 + (size_t)nblocks_max * sizeof(double) + 6 * 256;
  void* base = nullptr;
  lq_status st = lq_scratch(ctx, need, &base);
  if (st) return st;
  char* p = (char*)base;
  auto take = [&](size_t n) { p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); void* r = p; p += n; return r; };
  void* psi = take(vbytes);
  void* dchi = dSdchi ? dSdchi : take(vbytes);
  double* result = (double*)take(16);
  unsigned int* counter = (unsigned int*)take(sizeof(unsigned int));
  double* partials = (double*)take((size_t)nblocks_max * sizeof(double));
  LQ_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
  Reducer red{partials, counter, result, nblocks_max, 0 /*FIN_STORE*/, nullptr};

  // psi = D_oe chi
  DslashArgs d;
  d.U = U;
  d.in = chi;
  d.out = psi;
  d.out_parity = 1;
  d.nrhs = 1;
  d.vec_prec = vp;
  d.rhs_stride = U->Vh;
  st = launch_dslash(ctx, d, s);
  if (st) return st;
  // dS/dchi = 2 m^2 chi - 2 D_eo psi, and Re<chi, dS/dchi> = 2 S
  DslashArgs e = d;
  e.in = psi;
  e.out = dchi;
  e.out_parity = 0;
  e.w1 = chi;
  e.a1 = 2.0 * mass * mass;
  e.c = -2.0;
  e.reduce = RED_DOT;
  e.red = &red;
  st = launch_dslash(ctx, e, s);
  if (st) return st;
  if (dSdU || force_TA) {
    Geom G = make_geom(U);
    const int V = 2 * U->Vh;
    dim3 grid((V + kForceThreads - 1) / kForceThreads, 4);
    if (vp == LQ_F64) k_force<LQ_F64><<<grid, kForceThreads, 0, s>>>(U->data, U->blk_bytes, G, chi, psi, dSdU, force_TA);
    else k_force<LQ_F32><<<grid, kForceThreads, 0, s>>>(U->data, U->blk_bytes, G, chi, psi, dSdU, force_TA);
    LQ_CHECK_LAUNCH(ctx, "k_force");
  }
  if (S) {
    double two_s = 0.0;
    LQ_CUDA(ctx, cudaMemcpyAsync(&two_s, result, sizeof(double), cudaMemcpyDeviceToHost, s));
    LQ_CUDA(ctx, cudaStreamSynchronize(s));
    *S = 0.5 * two_s;
  }
  return LQ_OK;
}
