// Half-Dslash instances for f32 link storage (18- and 12-real): single-lattice and
// multi-lattice kernels.
#include "dslash_kernel.cuh"
#include "dslash_multi.cuh"

DslashLaunchFn dslash_fn_f32(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_F32, 12> : dslash_launch_gauge<LQ_F32, 18>;
}

MultiLaunchFn dslash_multi_fn_f32(int recon) {
  return recon == 12 ? multi_launch_gauge<LQ_F32, 12> : multi_launch_gauge<LQ_F32, 18>;
}

DslashTmaBlockFn dslash_tma_fn_f32(int recon) {
  return recon == 12 ? dslash_tma_block_of<LQ_F32, 12> : dslash_tma_block_of<LQ_F32, 18>;
}
