// Half-Dslash instances for f16 link storage (18- and 12-real).
#include "dslash_kernel.cuh"

DslashLaunchFn dslash_fn_f16(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_F16, 12> : dslash_launch_gauge<LQ_F16, 18>;
}
