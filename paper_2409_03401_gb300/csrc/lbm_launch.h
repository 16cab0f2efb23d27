// Host-side launch interface between the C-ABI (lbm_abi.cu) and the per-storage kernel
// translation units (lbm_step_<type>.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

#define LBM_NFIELDS_DEV 10
#define LBM_NRED_DEV 8

namespace lbm {

struct FieldPtrs { void* p[LBM_NFIELDS_DEV]; };

#define LBM_DECLARE_LAUNCHERS(SUFFIX)                                                                 \
    void launch_init_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow,                 \
                              const double*, const double*, const double*, cudaStream_t);             \
    void launch_phi_##SUFFIX(const DevParams&, const StateView&, int lat, bool odd, void* phi,        \
                             cudaStream_t);                                                           \
    void launch_step_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow, bool odd,       \
                              void* phi, cudaStream_t);                                               \
    void launch_fields_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow, bool odd,     \
                                void* phi, FieldPtrs, cudaStream_t);                                  \
    void launch_reduce_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow, bool odd,     \
                                void* phi, double* partials, int nblocks, cudaStream_t);

LBM_DECLARE_LAUNCHERS(f64)
LBM_DECLARE_LAUNCHERS(f32)
LBM_DECLARE_LAUNCHERS(f16)
LBM_DECLARE_LAUNCHERS(bf16)

}  // namespace lbm
