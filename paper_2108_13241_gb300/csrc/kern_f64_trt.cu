// kern_f64_trt.cu -- instantiates the step kernels with the two-relaxation-time
// collision for LBM_F64 storage (a translation unit of its own, compiled in
// parallel with the BGK instances of kern_f64.cu).
#include "lbm_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_STEP(LBM_F64, true)
} // namespace lbm
