// kern_f16s_trt.cu -- instantiates the step kernels with the two-relaxation-time
// collision for LBM_F16S storage (a translation unit of its own, compiled in
// parallel with the BGK instances of kern_f16s.cu).
#include "lbm_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_STEP(LBM_F16S, true)
} // namespace lbm
