// Half-Dslash instances for f64 link storage (18- and 12-real).
#include "dslash_kernel.cuh"

DslashLaunchFn dslash_fn_f64(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_F64, 12> : dslash_launch_gauge<LQ_F64, 18>;
}
