// Half-Dslash instances for f16 link storage (18- and 12-real): single-lattice and
// multi-lattice kernels.
#include "dslash_kernel.cuh"
#include "dslash_multi.cuh"

DslashLaunchFn dslash_fn_f16(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_F16, 12> : dslash_launch_gauge<LQ_F16, 18>;
}

MultiLaunchFn dslash_multi_fn_f16(int recon) {
  return recon == 12 ? multi_launch_gauge<LQ_F16, 12> : multi_launch_gauge<LQ_F16, 18>;
}

DslashTmaBlockFn dslash_tma_fn_f16(int recon) {
  return recon == 12 ? dslash_tma_block_of<LQ_F16, 12> : dslash_tma_block_of<LQ_F16, 18>;
}
