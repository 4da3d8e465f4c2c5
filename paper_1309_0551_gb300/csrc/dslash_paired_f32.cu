// Paired-layout multi-RHS half Dslash instances for f32 link storage (18- and 12-real).
#include "dslash_paired.cuh"

PairedLaunchFn dslash_paired_fn_f32(int recon) {
  return recon == 12 ? dslash_paired_launch<LQ_F32, 12> : dslash_paired_launch<LQ_F32, 18>;
}
