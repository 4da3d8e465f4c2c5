// Wilson hopping term instances: FP64 links (FP64 spinors).
#include "wilson_kernel.cuh"

WilsonLaunchFn wilson_fn_f64(int recon) {
  return recon == 12 ? wilson_launch<LQ_F64, 12> : wilson_launch<LQ_F64, 18>;
}
