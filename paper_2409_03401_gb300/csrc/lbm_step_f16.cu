// Coupled-step kernels instantiated for __half population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_LAUNCHERS(__half, f16)
}  // namespace lbm
