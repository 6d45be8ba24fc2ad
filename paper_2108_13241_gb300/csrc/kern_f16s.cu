// kern_f16s.cu -- instantiates the kernels and launchers of lbm_kernels.cuh for
// LBM_F16S storage (one translation unit per precision so they compile in parallel).
#include "lbm_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(LBM_F16S)
} // namespace lbm
