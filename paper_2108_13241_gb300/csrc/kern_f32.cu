// kern_f32.cu -- instantiates the kernels and launchers of lbm_kernels.cuh for
// LBM_F32 storage (one translation unit per precision so they compile in parallel).
#include "lbm_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(LBM_F32)
} // namespace lbm
