// Improved-Dslash instances for FP64 and FP32 links.
#include "dslash_improved.cuh"

ImprovedLaunchFn improved_fn_hi(lq_prec p) {
  return p == LQ_F64 ? improved_launch_gauge<LQ_F64> : improved_launch_gauge<LQ_F32>;
}
