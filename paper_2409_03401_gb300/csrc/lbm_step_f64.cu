// Coupled-step kernels instantiated for double population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_LAUNCHERS(double, f64)
}  // namespace lbm
