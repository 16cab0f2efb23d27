// Coupled-step kernels instantiated for float population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_LAUNCHERS(float, f32)
}  // namespace lbm
