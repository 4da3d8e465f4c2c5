// Leapfrog molecular dynamics around the fermion force, on the device end to end:
//   P += eps/2 F(U);  for k < n: U <- reunit(exp(eps P) U), P += (k < n-1 ? eps : eps/2) F(U)
// with F = TA(U G^dag) from dslash_force (H = -1/2 sum Tr P^2 + S, chi held fixed).  The
// links are re-packed into the caller's gauge object before each force evaluation
// (lq_gauge_repack: no allocation), the momentum update is scalar_mult_add_su3_matrix of
// Table 1 (su3_scalar_mult_add_batch) and the link update su3_exp_mul_batch.  Nothing is
// allocated per step and nothing synchronises but the final action, when it is asked for.
#include "lqcd_internal.cuh"
#include "tune.cuh"

extern "C" lq_status md_leapfrog(lq_context* ctx, lq_gauge* work, void* U, void* P, const void* chi, double mass,
                                 double eps, int nsteps, void* F, double* S, lq_stream stream) {
  if (!ctx) return LQ_ERR_INVALID_ARG;
  if (!work || !U || !P || !chi || !F) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "NULL argument");
  if (work->prec != LQ_F64 || work->recon != LQ_RECON_18)
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "md_leapfrog needs an LQ_F64, 18-real work gauge");
  if (nsteps < 1) return lq_fail(ctx, LQ_ERR_INVALID_ARG, "nsteps must be >= 1");
  if (!lq_aligned16(U) || !lq_aligned16(P) || !lq_aligned16(chi) || !lq_aligned16(F))
    return lq_fail(ctx, LQ_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
  const int64_t n = 4LL * 2 * work->Vh;   // links
  lq_status st;
  auto force = [&](double* s_out) -> lq_status {
    lq_status r = lq_gauge_repack(ctx, work, U, stream);
    if (r) return r;
    return dslash_force(ctx, work, mass, chi, nullptr, F, nullptr, s_out, stream);
  };
  if ((st = force(nullptr))) return st;
  if ((st = su3_scalar_mult_add_batch(ctx, P, F, P, 0.5 * eps, n, LQ_F64, stream))) return st;
  for (int k = 0; k < nsteps; ++k) {
    if ((st = su3_exp_mul_batch(ctx, P, U, U, eps, n, LQ_F64, stream))) return st;
    if ((st = force(k == nsteps - 1 ? S : nullptr))) return st;
    if ((st = su3_scalar_mult_add_batch(ctx, P, F, P, k < nsteps - 1 ? eps : 0.5 * eps, n, LQ_F64, stream)))
      return st;
  }
  return LQ_OK;
}
