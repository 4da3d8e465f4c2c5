// Half-Dslash instances for bf16 link storage (18- and 12-real): single-lattice and
// multi-lattice kernels.
#include "dslash_kernel.cuh"
#include "dslash_multi.cuh"

DslashLaunchFn dslash_fn_bf16(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_BF16, 12> : dslash_launch_gauge<LQ_BF16, 18>;
}

MultiLaunchFn dslash_multi_fn_bf16(int recon) {
  return recon == 12 ? multi_launch_gauge<LQ_BF16, 12> : multi_launch_gauge<LQ_BF16, 18>;
}

DslashTmaBlockFn dslash_tma_fn_bf16(int recon) {
  return recon == 12 ? dslash_tma_block_of<LQ_BF16, 12> : dslash_tma_block_of<LQ_BF16, 18>;
}
