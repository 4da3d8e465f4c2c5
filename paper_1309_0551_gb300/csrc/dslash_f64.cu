// Half-Dslash instances for f64 link storage (18- and 12-real): single-lattice and
// multi-lattice kernels.
#include "dslash_kernel.cuh"
#include "dslash_multi.cuh"

DslashLaunchFn dslash_fn_f64(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_F64, 12> : dslash_launch_gauge<LQ_F64, 18>;
}

MultiLaunchFn dslash_multi_fn_f64(int recon) {
  return recon == 12 ? multi_launch_gauge<LQ_F64, 12> : multi_launch_gauge<LQ_F64, 18>;
}
