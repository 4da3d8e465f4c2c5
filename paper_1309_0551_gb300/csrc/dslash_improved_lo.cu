// Improved-Dslash instances for bf16 and fp16 links.
#include "dslash_improved.cuh"

ImprovedLaunchFn improved_fn_lo(lq_prec p) {
  return p == LQ_BF16 ? improved_launch_gauge<LQ_BF16> : improved_launch_gauge<LQ_F16>;
}
