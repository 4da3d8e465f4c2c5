// Wilson hopping term instances: BF16 and FP16 links (FP32 spinors and arithmetic).
#include "wilson_kernel.cuh"

WilsonLaunchFn wilson_fn_16(lq_prec prec, int recon) {
  if (prec == LQ_BF16) return recon == 12 ? wilson_launch<LQ_BF16, 12> : wilson_launch<LQ_BF16, 18>;
  return recon == 12 ? wilson_launch<LQ_F16, 12> : wilson_launch<LQ_F16, 18>;
}
