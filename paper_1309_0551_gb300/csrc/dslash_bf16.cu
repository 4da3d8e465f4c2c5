// Half-Dslash instances for bf16 link storage (18- and 12-real).
#include "dslash_kernel.cuh"

DslashLaunchFn dslash_fn_bf16(int recon) {
  return recon == 12 ? dslash_launch_gauge<LQ_BF16, 12> : dslash_launch_gauge<LQ_BF16, 18>;
}
