// Paired-layout multi-RHS half Dslash instances for f16 link storage (18- and 12-real).
#include "dslash_paired.cuh"

PairedLaunchFn dslash_paired_fn_f16(int recon) {
  return recon == 12 ? dslash_paired_launch<LQ_F16, 12> : dslash_paired_launch<LQ_F16, 18>;
}
