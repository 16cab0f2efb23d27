// Coupled-step kernels instantiated for the 16-bit Store16 population storage (fixed point
// for g, IEEE FP16 for f and h; see Codec16 in lbm_device.cuh).
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_LAUNCHERS(Store16, f16)
}  // namespace lbm
