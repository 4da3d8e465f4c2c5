// Half-Dslash instances for f32 link storage (18- and 12-real).
#include "dslash_kernel.cuh"

DslashLaunchFn dslash_fn_f32(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_F32, 12> : dslash_launch_gauge<LQ_F32, 18>;
}
