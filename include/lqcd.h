/*
 * lqcd.h -- C ABI of the GB300 (sm_103a) staggered-fermion library.
 *
 * The library computes, on one GPU, the SU(3) link arithmetic that arXiv:1309.0551
 * ("Optimizing the performance of Lattice Gauge Theory simulations with Streaming SIMD
 * extensions") identifies as the bulk of a staggered lattice code's run time (Sec. 4:
 * the routines of Table 1 take 80-90% of it), in the form where it dominates: the
 * even/odd staggered Dslash and the conjugate-gradient solve it drives, plus the fermion
 * force.  Everything crossing this boundary is a plain pointer, size or enum.
 *
 * ---------------------------------------------------------------------------------------
 * Conventions (the paper states none of them; these are the library's):
 *   dims = {Lx, Ly, Lz, Lt}, every extent even and >= 2, periodic.  V = Lx*Ly*Lz*Lt,
 *   Vh = V/2.  lex = x + Lx*(y + Ly*(z + Lz*t)); parity = (x+y+z+t) & 1, even = 0;
 *   checkerboard index cb = lex >> 1 (the sites of one parity in lex order).
 *   Staggered phases eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z).
 *
 *   Gauge field, canonical:  complex128 U[4][V][3][3]  (U[mu][lex][row][col], the link
 *   from x to x+mu; interleaved re,im doubles; 16-byte aligned).
 *   Colour-vector field on one parity, canonical:  complex T v[nrhs][Vh][3] with T the
 *   vector precision (interleaved re,im; f64 = 2 doubles, f32 = 2 floats, bf16/f16 = 2
 *   16-bit values); 16-byte aligned base.
 *   SU(3) matrices for the batched routines: complex T A[n][3][3], row-major.
 *
 *   (D chi)(x) = sum_mu eta_mu(x) [ U_mu(x) chi(x+mu) - U_mu(x-mu)^dag chi(x-mu) ]
 *   (no factor 1/2).  M = m^2 - D_eo D_oe on even sites (Hermitian positive definite).
 *
 * Memory: every pointer argument named "device" is a device pointer on the context's
 * device, owned by the caller and only read or written during the call's stream work.
 * lq_gauge objects and the context's scratch space are owned by the library.  Every call
 * is asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 * stream) unless it says it synchronises.
 *
 * Errors: every entry point returns an lq_status; nothing aborts or traps.  On failure
 * lq_last_error(ctx) gives a message.  LQ_ERR_INVALID_ARG covers NULL pointers, odd or
 * non-positive extents, pointers not 16-byte aligned, unsupported precision pairs and
 * nrhs outside [1, 16].  A CUDA error is reported as LQ_ERR_CUDA with CUDA's string.
 * ---------------------------------------------------------------------------------------
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LQ_OK = 0,
  LQ_ERR_INVALID_ARG = 1,
  LQ_ERR_CUDA = 2,
  LQ_ERR_NOT_CONVERGED = 3,
  LQ_ERR_NUMERIC = 4,       /* NaN/Inf met (e.g. in a CG source or residual) */
  LQ_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  LQ_ERR_UNSUPPORTED = 6
} lq_status;

typedef enum { LQ_F64 = 0, LQ_F32 = 1, LQ_BF16 = 2, LQ_F16 = 3 } lq_prec;
typedef enum { LQ_RECON_18 = 18, LQ_RECON_12 = 12 } lq_recon;

typedef void* lq_stream;                 /* a cudaStream_t */
typedef struct lq_context lq_context;    /* device, scratch space, tuning cache, last error */
typedef struct lq_gauge lq_gauge;        /* packed links, library-owned device copy */

/* ----------------------------------------------------------------- context ---------- */

/* Create a context on CUDA device `device`.  *ctx receives the handle. */
lq_status lq_create(lq_context** ctx, int device);
/* Free a context and its scratch space (synchronises the device).  NULL is a no-op. */
lq_status lq_destroy(lq_context* ctx);
/* Message of the last failing call on this context ("" if none).  Valid until the next
 * call on the same context. */
const char* lq_last_error(const lq_context* ctx);
/* Name of a status code. */
const char* lq_status_string(lq_status s);
/* Synchronise `stream`, then report and clear the context's device status word: the
 * flags that bounded device waits set when they gave up since the last lq_sync.  Such a
 * wait exists in the batched SU(3) kernels (su3_*_batch), in the link-staging half
 * Dslash (dslash_eo and the solvers, when the tuner picks it) and in the single-RHS FP32
 * update of the mixed CG (cg_solve, cg_solve_noalloc), where one thread per block
 * waits, at most ~2^24 polls, for the TMA bulk copies that bring the block's operand slices
 * into shared memory; if they do not arrive, the block records the failure, waits once
 * more (bounded) so that it does not leave with copies in flight, and skips its work.
 * Those entry points are asynchronous and return LQ_OK at launch, so their outputs can
 * only be trusted after an lq_sync that returns LQ_OK (the CG solvers check the word
 * themselves).
 * Returns LQ_ERR_TIMEOUT if any wait gave up (outputs of the calls issued on this context
 * since the last lq_sync may be unwritten), LQ_ERR_CUDA for an error of the stream, LQ_OK
 * otherwise. */
lq_status lq_sync(lq_context* ctx, lq_stream stream);
/* Diagnostics for the error path above: synchronise `stream` and OR `flags` into the
 * context's device status word from the host, exactly as a device wait that gave up
 * would; the next lq_sync reports LQ_ERR_TIMEOUT.  No kernel runs. */
lq_status lq_inject_status(lq_context* ctx, unsigned int flags, lq_stream stream);
/* Self-test of the bounded device wait: one block of the batched mat-vec kernel arms its
 * mbarrier for its operand bytes but issues no copy, so its (short, ~2^10 polls) wait runs
 * out with nothing in flight; the block sets the status flag and returns.  The next
 * lq_sync returns LQ_ERR_TIMEOUT.  Asynchronous on `stream`. */
lq_status lq_selftest_wait_timeout(lq_context* ctx, lq_stream stream);

/* Autotuning of launch shapes (threads per block, right-hand sides per thread, threads per
 * site).  mode 0: off, fixed defaults.  mode 1 (the default, unless the environment sets
 * LQCD_TUNE=0): each new shape key is tuned on its first call by timing every candidate
 * as a lone launch after an L2 flush; among the candidates within 3% of the fastest the
 * one with the least redundant work wins.  mode 2: the same, with a 15% margin -- for
 * callers that keep several independent launches in flight (streams, graphs), where a
 * launch's own parallelism matters less than its instruction count.  Tuning must not
 * happen during stream capture: make one uncaptured call with the same shapes first.  The
 * environment variable LQCD_DSLASH_SHAPE="block,rhs_tile,threads_per_site" forces one
 * shape for every Dslash launch it fits (block 64..256, a multiple of 32).  threads_per_site
 * 1, 2 or 4 selects the split-site kernel; 8 the rhs-per-warp multi-RHS kernel (rhs_tile =
 * right-hand sides per block); 16 the link-staging kernel (rhs_tile 1); 32 the paired-layout
 * kernel of dslash_eo_paired (rhs_tile = pairs of right-hand sides per thread: 1, 2, 4). */
lq_status lq_set_tuning(lq_context* ctx, int mode);
/* Persist the tuning table in the file `path` (NULL or "" stops persisting): the entries
 * the file holds for this device (same name and SM count) are loaded now, without
 * replacing shapes already in the table, and the table is saved to the file each time a
 * new shape is tuned.  Two processes sharing the file then launch every kernel with the
 * same shape -- the same summation order in every reduction, hence the same CG iterates
 * and iteration counts.  lq_create does this itself when the environment variable
 * LQCD_TUNE_CACHE names a file.  Processes that tune concurrently may overwrite each
 * other's new entries (the last save wins); a lost entry is tuned again. */
lq_status lq_set_tune_cache(lq_context* ctx, const char* path);
/* Write the tuning table (one line per key: key, chosen block, rhs tile, microseconds)
 * into buf (NUL-terminated, truncated to len).  *needed receives the full length + 1. */
lq_status lq_tune_report(const lq_context* ctx, char* buf, size_t len, size_t* needed);

/* Measure the device's FP64 FMA rate (GFLOP/s, 2 flops per FMA) with a kernel of
 * independent FMA chains on every SM, timed with CUDA events (best of three after a
 * warm-up run; synchronises the device's legacy stream).  GB300 runs FP64 far below its
 * FP32 rate: the FP64 kernels here are bound by this pipe, and this figure is the
 * denominator of their roofline.  The paper has no counterpart (its peak figure is the
 * Pentium 4's, Sec. 2). */
lq_status lq_fp64_fma_rate(lq_context* ctx, double* gflops);

/* ------------------------------------------------------------------- gauge ---------- */

/* Pack a canonical complex128 gauge field (device, U[4][V][3][3]) into the library's
 * internal layout with storage precision `prec` and `recon` reals per link.
 *   Internal layout: structure of arrays per (direction, parity) block, sites in
 *   checkerboard order, the reals of a link split into "planes" of 16-byte (or smaller)
 *   chunks so that each thread reads its link with few wide coalesced loads.  Recon 12
 *   keeps rows 0 and 1; row 2 is rebuilt as conj(row0 x row1) in registers (exact for
 *   SU(3) links up to rounding).  Reduced precisions round each real once (to nearest,
 *   ties to even) from FP64.
 * The gauge object keeps no reference to U. */
lq_status lq_gauge_pack(lq_context* ctx, const int dims[4], const void* U_canon,
                        lq_prec prec, lq_recon recon, lq_gauge** out, lq_stream stream);
lq_status lq_gauge_free(lq_context* ctx, lq_gauge* g);
/* Re-pack a canonical complex128 field (device, [4][V][3][3], same lattice) into the
 * existing gauge object g, keeping its precision and recon: no allocation, asynchronous on
 * `stream` (work already queued that reads g must be ordered before it by the caller). */
lq_status lq_gauge_repack(lq_context* ctx, lq_gauge* g, const void* U_canon, lq_stream stream);
/* Bytes of device memory the packed field occupies (for bandwidth accounting). */
lq_status lq_gauge_info(const lq_gauge* g, int dims[4], lq_prec* prec, lq_recon* recon,
                        size_t* bytes);

/* -------------------------------------------------------- SU(3) batches ------------- */

/* C[i] = op(A[i]) op(B[i]) for i < n; op = adjoint when adjA / adjB is 1.  Table 1:
 * mult_su3_nn (0,0), mult_su3_an (1,0), mult_su3_na (0,1).  198 flops per product.
 * A, B, C: device, complex [n][3][3] of `prec` (LQ_F64 or LQ_F32); C must not overlap
 * A or B.  n = 0 is a no-op. */
lq_status su3_mul_batch(lq_context* ctx, const void* A, const void* B, void* C, int64_t n,
                        int adjA, int adjB, lq_prec prec, lq_stream stream);

/* c[i] = op(A[i]) b[i]; op = adjoint when adj = 1.  Table 1: mult_su3_mat_vec (adj 0) and
 * mult_adj_su3_mat_vec (adj 1; its first component is Eqs. (1.1)-(2.3)).  66 flops each.
 * A: device complex [n][3][3]; b, c: device complex [n][3]; prec LQ_F64 or LQ_F32. */
lq_status su3_matvec_batch(lq_context* ctx, const void* A, const void* b, void* c,
                           int64_t n, int adj, lq_prec prec, lq_stream stream);

/* su3_matvec_batch with any storage format: c[i] = op(A[i]) b[i] (Table 1:
 * mult_su3_mat_vec, adj 0, and mult_adj_su3_mat_vec, adj 1, whose first component is
 * Eqs. (1.1)-(2.3)); 66 flops each.
 *   A: device, complex [n][3][3] of mat_prec with recon LQ_RECON_18, or complex [n][2][3]
 *      (rows 0 and 1 only) with LQ_RECON_12: row 2 is rebuilt as conj(row0 x row1), exact
 *      for SU(3) matrices up to rounding.  16-bit complex values are (re, im) pairs of
 *      bfloat16 / binary16 (4 bytes per complex).
 *   b, c: device complex [n][3] of vec_prec; c must not overlap A or b.
 *   Pairs: LQ_F64 matrices with LQ_F64 vectors (FP64 arithmetic); LQ_F32 / LQ_BF16 /
 *   LQ_F16 matrices with LQ_F32 / LQ_BF16 / LQ_F16 vectors (FP32 arithmetic, one rounding
 *   of each output real).  n = 0 is a no-op. */
lq_status su3_matvec_batch_ex(lq_context* ctx, const void* A, const void* b, void* c, int64_t n, int adj,
                              lq_prec mat_prec, lq_recon recon, lq_prec vec_prec, lq_stream stream);

/* c[i] = op(A[i]) h[i] for half Wilson vectors h (two colour vectors, i.e. two spin
 * components); op = adjoint when adj = 1.  Table 1: mult_su3_mat_hwvec (adj 0) and
 * mult_adj_su3_mat_hwvec (adj 1).  132 flops each.
 * A: device complex [n][3][3]; h, c: device complex [n][2][3]; prec LQ_F64 or LQ_F32;
 * c must not overlap A or h. */
lq_status su3_mat_hwvec_batch(lq_context* ctx, const void* A, const void* h, void* c,
                              int64_t n, int adj, lq_prec prec, lq_stream stream);

/* C[i] = A[i] + s B[i] (Table 1: scalar_mult_add_su3_matrix), e.g. the momentum update
 * P <- P + s F of a molecular-dynamics step.  A, B, C: device complex [n][3][3] of `prec`
 * (LQ_F64 or LQ_F32); C may be A or B. */
lq_status su3_scalar_mult_add_batch(lq_context* ctx, const void* A, const void* B, void* C, double s,
                                    int64_t n, lq_prec prec, lq_stream stream);

/* out[i] = reunit(exp(eps P[i]) U[i]) for traceless anti-Hermitian P (the link update of a
 * molecular-dynamics step; the paper does not write it down).  exp by scaling and
 * squaring of a Taylor polynomial (degree 12 in FP64, 7 in FP32, argument scaled to a
 * row-sum norm <= 1/4); reunit orthonormalises rows 0, 1 and sets row 2 = conj(r0 x r1).
 * P, U, out: device complex [n][3][3] of `prec` (LQ_F64 or LQ_F32); out may be U. */
lq_status su3_exp_mul_batch(lq_context* ctx, const void* P, const void* U, void* out, double eps,
                            int64_t n, lq_prec prec, lq_stream stream);

/* ------------------------------------------------------------------ Dslash ---------- */

/* Half Dslash: out = D in restricted to the sites of parity `out_parity`, `in` living on
 * the other parity (out_parity 1: D_oe, 0: D_eo), for nrhs right-hand sides that share
 * each loaded link.  570 flops per output site and right-hand side.
 *   in, out: device, canonical vector fields [nrhs][Vh][3] of `vec_prec`; must not overlap.
 *   Precision pairs: an LQ_F64 gauge needs LQ_F64 vectors (FP64 arithmetic); an LQ_F32,
 *   LQ_BF16 or LQ_F16 gauge takes LQ_F32, LQ_BF16 or LQ_F16 vectors (FP32 arithmetic and
 *   accumulation, one rounding at the store).  16-bit vectors carry no scale factor: their
 *   values must lie in the format's range.
 *   nrhs in [1, 16]. */
lq_status dslash_eo(lq_context* ctx, const lq_gauge* U, const void* in, void* out,
                    int out_parity, int nrhs, lq_prec vec_prec, lq_stream stream);

/* The half Dslash of dslash_eo applied to nlat lattices (at most 16, sizes may differ) in
 * ONE persistent launch: the work is cut into (lattice, rhs tile, site block) tiles that a
 * grid of about one wave of resident blocks walks in a fixed order, so that many small
 * lattices, or several independent fields, fill the GPU together.  Tile shapes are
 * autotuned per lattice set.
 *   U[l]: gauges of one storage format; in[l], out[l]: device, [nrhs][Vh_l][3] vectors.
 *   Precision pairs: LQ_F64 links with LQ_F64 vectors; LQ_F32/LQ_BF16/LQ_F16 links with
 *   LQ_F32 vectors. */
lq_status dslash_eo_multi(lq_context* ctx, int nlat, const lq_gauge* const* U, const void* const* in,
                          void* const* out, int out_parity, int nrhs, lq_prec vec_prec,
                          lq_stream stream);

/* Paired colour-planar FP32 layout for several right-hand sides.  Right-hand sides are
 * taken two at a time: pair p = 0 .. npair-1 (npair = (nrhs + 1) / 2) is three colour
 * planes of Vh float4, element [p][c][site] = (Re v_2p, Re v_2p+1, Im v_2p, Im v_2p+1) of
 * colour c at that site; npair * 3 * Vh * 16 bytes.  With odd nrhs the second half of the
 * last pair is padding.  It is the layout of dslash_eo_paired.
 *
 * lq_vec_pair: canonical complex64 [nrhs][Vh][3] (in) -> paired (out); the padding half is
 * written as zero.  lq_vec_unpair: paired (in) -> canonical (out); the padding half is not
 * read.  Element copies, bit-exact.  Both device pointers 16-byte aligned, not overlapping;
 * Vh >= 1, nrhs in [1, 16].  Asynchronous on `stream`. */
lq_status lq_vec_pair(lq_context* ctx, int Vh, int nrhs, const void* in, void* out, lq_stream stream);
lq_status lq_vec_unpair(lq_context* ctx, int Vh, int nrhs, const void* in, void* out, lq_stream stream);

/* The half Dslash of dslash_eo (Eqs. (1.1)-(2.3) summed over the eight hops) for nrhs
 * right-hand sides held in the paired layout (FP32 vectors and arithmetic; LQ_F32,
 * LQ_BF16 or LQ_F16 links, 12 or 18 reals).  Each thread applies every loaded link element
 * to two right-hand sides with one packed FP32x2 FMA, and loads each colour of a pair with
 * one 16-byte access.  Same operator as dslash_eo with LQ_F32 vectors; the FMA order
 * differs, so results agree within FP32 rounding, not bit for bit.
 *   in, out: device, paired fields of U->Vh sites; must not overlap.  nrhs in [1, 16].
 *   Errors: LQ_ERR_INVALID_ARG for an LQ_F64 gauge, NULL or misaligned pointers, a bad
 *   parity or nrhs. */
lq_status dslash_eo_paired(lq_context* ctx, const lq_gauge* U, const void* in, void* out,
                           int out_parity, int nrhs, lq_stream stream);

/* Improved staggered half Dslash with one-hop ("fat") links F and three-hop ("long",
 * Naik) links L -- the operator of the improved staggered application the paper times
 * (Table 4; the paper does not write it down):
 *   out(x) = sum_mu eta_mu(x) [ F_mu(x) in(x+mu) - F_mu(x-mu)^dag in(x-mu)
 *                              + L_mu(x) in(x+3mu) - L_mu(x-3mu)^dag in(x-3mu) ]
 * 1146 flops per output site and rhs.  fat, lng: lq_gauge objects of one lattice packed
 * with recon 18 and the same precision (fat links are not unitary, long links carry their
 * coefficient; the smearing that makes F is the caller's).  in, out, nrhs, vec_prec: as
 * for dslash_eo. */
lq_status dslash_eo_improved(lq_context* ctx, const lq_gauge* fat, const lq_gauge* lng, const void* in,
                             void* out, int out_parity, int nrhs, lq_prec vec_prec, lq_stream stream);

/* Naik links L_mu(x) = coeff * U_mu(x) U_mu(x+mu) U_mu(x+2mu) (two mult_su3_nn per link,
 * Table 1), FP64.  U_canon, L_canon: device complex128 [4][V][3][3] (must not overlap).
 * Pack L with lq_gauge_pack(..., LQ_RECON_18, ...) for dslash_eo_improved. */
lq_status lq_long_links(lq_context* ctx, const int dims[4], const void* U_canon, double coeff,
                        void* L_canon, lq_stream stream);

/* Wilson hopping term on one parity (the Wilson Dslash), the operator Table 1's half
 * Wilson vector routines serve (the paper does not write it down):
 *   out(x) = sum_mu [ (1 - s gamma_mu) U_mu(x) in(x+mu) + (1 + s gamma_mu) U_mu(x-mu)^dag in(x-mu) ]
 * for x of parity `out_parity`, `in` on the other parity; s = `sign` (+1, or -1 for the
 * adjoint: gamma_5 D gamma_5); gamma matrices in the DeGrand-Rossi (chiral) basis,
 * gamma_5 = diag(1, 1, -1, -1); periodic; no mass or kappa factor.  Each hop projects
 * the neighbour spinor to a half Wilson vector, multiplies it by the link
 * (mult_su3_mat_hwvec / mult_adj_su3_mat_hwvec) and rebuilds the other two spin
 * components: 1320 flops per output site and rhs.
 *   U: any packed gauge (the staggered phases are not in the links).
 *   in, out: device spinor fields [nrhs][Vh][4][3] complex, [spin][colour]; LQ_F64 for
 *   LQ_F64 links, LQ_F32 for LQ_F32 / LQ_BF16 / LQ_F16 links (FP32 arithmetic); must not
 *   overlap.  nrhs in [1, 16]. */
lq_status dslash_wilson_eo(lq_context* ctx, const lq_gauge* U, const void* in, void* out,
                           int out_parity, int nrhs, lq_prec vec_prec, int sign, lq_stream stream);

/* -------------------------------------------------- t-split domain decomposition --- */
/* A lattice (Lx, Ly, Lz, Lt) cut in t into P sub-domains of Lt/P (even) slices, one per
 * process or GPU: the method's parallel mode (Table 4's parallel runs; the communication
 * term of the timing model in Sec. 4), which the paper does not spell out.  Sub-domain k
 * is packed as a lattice of its own, (Lx, Ly, Lz, Lt/P), from the slices
 * [k Lt/P, (k+1) Lt/P) of the canonical fields (contiguous ranges: U[mu][t0 Vs : ...],
 * one-parity vectors [t0 Vs/2 : ...], Vs = Lx Ly Lz).  Its half Dslash needs one face from
 * each t neighbour (cyclic): the input on the next sub-domain's first slice and on the
 * previous one's last slice -- the first / last Vs/2 sites of their own arrays, complex
 * [nrhs][Vs/2][3] -- and, once, the previous sub-domain's U_t on its last slice.  The
 * caller moves faces (NCCL send/recv, peer copies, ...) into buffers of its own device. */

/* Attach the ghost links of a sub-domain to its gauge: Ut_ghost = device complex128
 * [Vs][3][3], the previous sub-domain's U_t on its last slice in lex order within the slice
 * (U_prev[3][(Lt/P - 1) Vs : Lt/P Vs]).  Stored in g's precision and recon (allocated on
 * the first call, freed with g).  Asynchronous on stream. */
lq_status lq_gauge_set_halo(lq_context* ctx, lq_gauge* g, const void* Ut_ghost, lq_stream stream);

/* Half Dslash of a sub-domain: out = a1 w1 + c D in, D as in dslash_eo on the local
 * lattice except that the t hops leaving it read ghost_fwd (forward hops from the last
 * slice: the next sub-domain's first-slice face) and ghost_bwd with the ghost links
 * (backward hops from the first slice: the previous sub-domain's last-slice face), each
 * device complex [nrhs][Vs/2][3] of vec_prec.  With P = 1 (each sub-domain its own
 * neighbour) it is dslash_eo.  U: a gauge with lq_gauge_set_halo done; vec_prec LQ_F64 for
 * LQ_F64 links, LQ_F32 otherwise; w1 nullable (then a1 is ignored); out must not be in or
 * w1.  One thread per output site and rhs.  570 flops per site and rhs. */
lq_status dslash_eo_halo(lq_context* ctx, const lq_gauge* U, const void* in, const void* ghost_bwd,
                         const void* ghost_fwd, void* out, int out_parity, int nrhs, lq_prec vec_prec,
                         double a1, const void* w1, double c, lq_stream stream);

/* Vector kernels for a solver driven by the caller (the t-split CG, whose inner products
 * are summed across sub-domains between launches): on n complex values of prec (LQ_F64 or
 * LQ_F32), y = a x + b y (y may be x) ... */
lq_status lq_vec_axpby(lq_context* ctx, int64_t n, double a, const void* x, double b, void* y, lq_prec prec,
                       lq_stream stream);
/* ... and *result (device double) = Re<x, y>, each product and the sum in FP64 (fixed
 * order for a given n: deterministic).  Uses the context's scratch space. */
lq_status lq_vec_dot(lq_context* ctx, int64_t n, const void* x, const void* y, lq_prec prec, double* result,
                     lq_stream stream);

/* ---------------------------------------------------------------------- CG ---------- */

typedef struct {
  double tol;          /* stop when ||b - M x|| / ||b|| <= tol, M in FP64 (true residual) */
  int maxiter;         /* inner iterations, all right-hand sides together */
  int reliable_every;  /* mixed precision: FP64 residual replacement at least this often */
  double delta;        /* mixed precision: ... or when ||r_lo|| < delta * ||r|| at the last one */
  int check_every;     /* iterations per device-resident block between host checks (graph) */
} lq_cg_params;

typedef struct {
  int iters;              /* inner iterations until this right-hand side converged */
  int reliable_updates;   /* FP64 residual replacements (mixed precision) */
  double true_rel_resid;  /* ||b - M x|| / ||b|| recomputed in FP64 at exit */
  double seconds;         /* wall time of the whole call */
} lq_cg_stats;

/* Solve M x = b, M = m^2 - D_eo D_oe on even sites, by conjugate gradient from x = 0.
 *   U_hi: LQ_F64 gauge (recon 18 or 12): defines M and every true residual.
 *   U_lo: NULL -> plain FP64 CG.  Otherwise an LQ_F32 / LQ_BF16 / LQ_F16 gauge of the same
 *         lattice: the inner iteration applies M with those links, keeps its vectors in
 *         FP32 with FP64 inner products, and replaces its residual by the FP64 true
 *         residual (reliable update) every params->reliable_every iterations, or when it
 *         fell below params->delta times the last replaced one, or on apparent convergence.
 *         The search direction is kept across a replacement, with the Polak-Ribiere
 *         beta = max(0, Re<r_new, r_new - r_k>) / ||r_k||^2 (r_k: the residual that
 *         entered the last iteration; equal to ||r_new||^2 / ||r_k||^2 in exact
 *         arithmetic), the choice of flexible CG for an operator that differs from the
 *         one the residual is corrected with.  The FP64 solve restarts the same way when
 *         its iterated residual meets tol but its true residual does not.
 *   b, x: device complex128 [nrhs][Vh][3]; x is overwritten.  nrhs in [1, 16].
 *   stats: host array of nrhs entries (may be NULL).
 *   With U_lo and nrhs >= 2 the inner vectors are kept in the paired colour-planar layout
 *   of dslash_eo_paired (converted to and from the canonical layout only at the reliable
 *   updates); the environment variable LQCD_CG_PAIRED=0 keeps them canonical.  Both reach
 *   the same tolerance; iterates differ by FP32 rounding order.
 * Synchronises `stream` at each check (every check_every iterations).  Returns
 * LQ_ERR_NOT_CONVERGED if maxiter was reached (stats filled in), LQ_ERR_NUMERIC if b or a
 * residual holds NaN/Inf, LQ_ERR_TIMEOUT if the context's device status word holds a
 * bounded wait that gave up (see lq_sync; the word is then cleared). */
lq_status cg_solve(lq_context* ctx, const lq_gauge* U_hi, const lq_gauge* U_lo, double mass,
                   const void* b, void* x, int nrhs, const lq_cg_params* params,
                   lq_cg_stats* stats, lq_stream stream);

/* ------------------------------------------------------------------- force ---------- */

/* Gradients of the pseudofermion action S = Re chi^dag M chi = m^2 ||chi||^2 + ||D_oe chi||^2
 * (M = m^2 - D_eo D_oe, chi on the even sites).  The paper lists the building blocks
 * (Table 1: su3_projector for the outer products, mult_su3_na for U G^dag) but not the
 * force itself; conventions are the library's:
 *   psi = D_oe chi (recomputed on every call);
 *   dSdchi = 2 M chi  -- the gradient with respect to (Re chi, Im chi), packed as complex;
 *   dSdU[mu][lex] = G = 2 Z^dag with Z = eta_mu(y) chi(y+mu) psi(y)^dag for odd y and
 *     Z = -eta_mu(y) psi(y+mu) chi(y)^dag for even y, so that dS = Re sum Tr(G^dag dU);
 *   force_TA[mu][lex] = TA(U G^dag), TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6, so that
 *     d/de S(exp(e X) U) = Tr(X F) for every traceless anti-Hermitian X.
 *   U: 18-real gauge, LQ_F64 or LQ_F32; chi (device, [Vh][3]) and every output use the
 *   same precision (complex128 or complex64).  dSdU and force_TA are canonical gauge-shaped
 *   [4][V][3][3]; any of dSdU, force_TA, dSdchi, S may be NULL.  S (host) makes the call
 *   synchronise the stream.  Cost per call: two half Dslash and one pass over the links. */
lq_status dslash_force(lq_context* ctx, const lq_gauge* U, double mass, const void* chi,
                       void* dSdU, void* force_TA, void* dSdchi, double* S, lq_stream stream);

/* Leapfrog molecular dynamics for H = -1/2 sum Tr(P^2) + S(U), S = Re chi^dag M chi with chi
 * held fixed (the integrator around the fermion force; the paper does not write it down):
 *   P += eps/2 F(U);  then nsteps times: U = reunit(exp(eps P) U), P += eps F(U), the last
 *   momentum step being eps/2 -- with F = TA(U G^dag) of dslash_force, the momentum update
 *   scalar_mult_add_su3_matrix (Table 1) and the link update of su3_exp_mul_batch.
 *   work: an LQ_F64, 18-real gauge object of the lattice, owned by the caller: the links
 *         are re-packed into it (lq_gauge_repack) before every force evaluation.
 *   U, P: device complex128 [4][V][3][3], updated in place; chi: device complex128 [Vh][3];
 *   F: device complex128 [4][V][3][3] scratch for the force (caller-owned).
 *   S: host, nullable: the action at the final links (the call then synchronises stream).
 * No allocation per step (the force's work vectors live in the context's scratch space,
 * grown on first use); every step runs in the library's kernels on `stream`. */
lq_status md_leapfrog(lq_context* ctx, lq_gauge* work, void* U, void* P, const void* chi, double mass, double eps,
                      int nsteps, void* F, double* S, lq_stream stream);

/* Batched solve of nlat independent lattices (uneven sizes allowed, at most 16), each with
 * nrhs right-hand sides and its own mass: every system (lattice, rhs) runs the cg_solve
 * iteration, but each phase of an iteration is ONE launch over all lattices -- a
 * persistent multi-lattice Dslash kernel walking (lattice, rhs tile, site block) tiles
 * (per thread, or spread over the warps of a block with the links shared), and
 * persistent vector kernels walking (lattice, rhs, site block) tiles -- and the iteration
 * block is captured once as a CUDA graph.  Tile shapes (sites per block, right-hand sides
 * per thread, threads per site) come from the autotuner, keyed by the lattice set.
 *   U_hi[l]: LQ_F64 gauges (all the same recon).  U_lo: NULL (FP64 solve) or an array of
 *   reduced-precision gauges of one format (mixed precision as in cg_solve).  Reliable
 *   updates are taken per lattice: when one system of a lattice is due, all of that
 *   lattice's right-hand sides take it (as in cg_solve), and the FP64 work of the other
 *   lattices is skipped.
 *   mass[l], b[l], x[l]: host arrays of nlat entries; b[l], x[l] are device complex128
 *   [nrhs][Vh_l][3].  stats: host array of nlat * nrhs entries, [l * nrhs + rhs].
 * Paper: the batching pattern is not in the paper; each system is the CG of cg_solve. */
lq_status cg_solve_batched(lq_context* ctx, int nlat, const lq_gauge* const* U_hi,
                           const lq_gauge* const* U_lo, const double* mass, const void* const* b,
                           void* const* x, int nrhs, const lq_cg_params* params,
                           lq_cg_stats* stats, lq_stream stream);

/* Allocation-free variant of cg_solve.  The paper has no counterpart; this entry point
 * exists for callers that cannot allocate GPU memory when they solve -- for example code
 * running inside a host framework or plugin that forbids cudaMalloc/cudaFree on its
 * threads, or a loop under a fixed memory budget that must not grow or synchronise the
 * device through an allocation.
 *   Same arguments, results and statuses as cg_solve.  Its scratch space (work vectors,
 *   per-rhs scalars, reduction partials) is a fixed 32 MiB array inside the library
 *   image, so every GPU that loads the library holds those 32 MiB until the process
 *   exits.  It calls no cudaMalloc, cudaFree or cudaMallocHost, and creates no stream,
 *   event or graph: the solve runs as plain kernel launches on `stream`, synchronising it
 *   at each check.  Launch shapes come from the context's tuning table when an earlier
 *   call (e.g. cg_solve with the same gauges) filled it, else fixed defaults.
 *   Limit: (4 inner vectors, 5 with U_lo) * nrhs * Vh * 48 bytes (24 with U_lo) + 2 FP64
 *   vectors of nrhs * Vh * 48 bytes + 3 * nrhs * Vh/16 * 8 + nrhs * 256 bytes of partials
 *   must fit in 32 MiB (e.g. a 16^4 lattice with one right-hand side); larger problems get
 *   LQ_ERR_INVALID_ARG with a message naming the sizes.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   and caches it; make that first call before any stream capture.
 *   All calls share the one array and each leaves its contents behind (the call clears
 *   what must start at zero): calls whose GPU work overlaps -- on different streams,
 *   threads or contexts of the same device -- race on it and give wrong results. */
lq_status cg_solve_noalloc(lq_context* ctx, const lq_gauge* U_hi, const lq_gauge* U_lo, double mass,
                           const void* b, void* x, int nrhs, const lq_cg_params* params,
                           lq_cg_stats* stats, lq_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
