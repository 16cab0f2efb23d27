// Host-side launch interface between the C-ABI (lbm_abi.cu) and the per-storage kernel
// translation units (lbm_step_<type>.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

#define LBM_NFIELDS_DEV 10
#define LBM_NRED_DEV 10

namespace lbm {

struct FieldPtrs { void* p[LBM_NFIELDS_DEV]; };

// streaming modes (see lbm_kernels.cuh)
constexpr int kModeAAEven = 0, kModeAAOdd = 1, kModePull = 2;

#define LBM_DECLARE_LAUNCHERS(SUFFIX)                                                                   \
    void launch_init_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow, bool pull,         \
                              const double*, const double*, const double*, cudaStream_t);                \
    void launch_phi_##SUFFIX(const DevParams&, const StateView&, int lat, int mode, void* phi,           \
                             cudaStream_t);                                                              \
    void launch_plane_phi_##SUFFIX(const DevParams&, const StateView&, int lat, int mode, int z, void* out, \
                                   cudaStream_t);                                                        \
    void launch_step_##SUFFIX(const DevParams&, const StateView&, const StateView&, int lat, bool flow, \
                              int mode, void* phi, cudaStream_t);                                        \
    void launch_fused_##SUFFIX(const DevParams&, const StateView&, const StateView&, int zchunk,        \
                               cudaStream_t);                                                            \
    void launch_fields_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow, int mode,        \
                                void* phi, FieldPtrs, cudaStream_t);                                     \
    void launch_reduce_##SUFFIX(const DevParams&, const StateView&, int lat, bool flow, int mode,        \
                                void* phi, void* bits, double* partials, int nblocks, cudaStream_t);

void launch_adjoint_step(const DevParams&, const StateView&, int storage, int lat, bool odd, const void* lam_next,
                         void* lam, double* partials, cudaStream_t);
void launch_adjoint_seed(const DevParams&, const StateView&, int storage, int lat, bool odd, const void* phib,
                         const void* muAb, const void* muBb, void* lam, double* partials, cudaStream_t);
void launch_adjoint_init(const DevParams&, int storage, int lat, const double* phi0, const double* cA0,
                         const double* cB0, const void* lam, double* phi0b, double* partials, cudaStream_t);
void launch_theta_final(const double* partials, int rows, double* out, cudaStream_t);
long long adjoint_rows(const DevParams& P);
int adjoint_ntheta();

LBM_DECLARE_LAUNCHERS(f64)
LBM_DECLARE_LAUNCHERS(f32)
LBM_DECLARE_LAUNCHERS(f16)
LBM_DECLARE_LAUNCHERS(bf16)

}  // namespace lbm
