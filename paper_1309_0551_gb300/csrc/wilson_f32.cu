// Wilson hopping term instances: FP32 links (FP32 spinors).
#include "wilson_kernel.cuh"

WilsonLaunchFn wilson_fn_f32(int recon) {
  return recon == 12 ? wilson_launch<LQ_F32, 12> : wilson_launch<LQ_F32, 18>;
}
