// Coupled-step kernels instantiated for __nv_bfloat16 population storage.
#include "lbm_kernels.cuh"

namespace lbm {
LBM_DEFINE_LAUNCHERS(__nv_bfloat16, bf16)
}  // namespace lbm
