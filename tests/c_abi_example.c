/* A plain C caller of the library: no Python, no torch. It allocates the state and scratch
 * with cudaMalloc, builds a droplet of phase 1 at rest in a wall-bounded box, runs the coupled
 * step with flow through include/lbm.h, and checks what the method fixes exactly: sum c^A,
 * sum c^B and sum p_h do not change (Eqs. 40, 52), sum g changes by exactly the sum of the
 * phase-field source (Eqs. 46-49), phi stays in [0, 1] and every moment stays finite.
 * Prints one line and returns 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "lbm.h"

#define CHECK(cond, msg)                                            \
    do {                                                            \
        if (!(cond)) {                                              \
            fprintf(stderr, "FAILED: %s\n", msg);                   \
            return 1;                                               \
        }                                                           \
    } while (0)

int main(void) {
    lbm_params p = {0};
    p.nx = 40; p.ny = 36; p.nz = 28;
    p.lattice = LBM_D3Q7; p.flow = 1; p.storage = LBM_F32; p.wall_z = 1;
    p.W = 3.0; p.lambda = 155.95; p.M_phi = 0.12;
    p.c_eq[0][0] = 0.3; p.c_eq[0][1] = 0.3; p.c_eq[1][0] = 0.4; p.c_eq[1][1] = 0.4;
    p.M[0][0] = 0.1; p.M[0][1] = 0.08; p.M[1][0] = 0.1; p.M[1][1] = 0.08;
    p.nu = 0.1; p.sigma = 1e-3; p.g[2] = -1e-5;
    p.collision = LBM_BGK;
    const size_t n = (size_t)p.nx * p.ny * p.nz;
    const size_t sb = lbm_state_bytes(&p), wb = lbm_work_bytes(&p);
    CHECK(sb > 0 && wb > 0, lbm_last_error(NULL));

    double* h = (double*)malloc(3 * n * sizeof(double));
    CHECK(h != NULL, "host allocation");
    for (int z = 0; z < p.nz; ++z)
        for (int y = 0; y < p.ny; ++y)
            for (int x = 0; x < p.nx; ++x) {
                const size_t i = ((size_t)z * p.ny + y) * p.nx + x;
                const double r = sqrt((x - 19.5) * (x - 19.5) + (y - 17.5) * (y - 17.5) + (z - 13.5) * (z - 13.5));
                const double phi = 0.5 * (1.0 + tanh(2.0 * (8.0 - r) / p.W));   /* Eq. 13 */
                h[i] = phi;
                h[n + i] = phi >= 0.5 ? 0.4 : 0.302;                          /* c^A */
                h[2 * n + i] = phi >= 0.5 ? 0.4 : 0.302;                      /* c^B */
            }
    void *state = NULL, *work = NULL, *init = NULL, *phi_out = NULL;
    CHECK(cudaMalloc(&state, sb) == cudaSuccess, "cudaMalloc state");
    CHECK(cudaMalloc(&work, wb) == cudaSuccess, "cudaMalloc work");
    CHECK(cudaMalloc(&init, 3 * n * sizeof(double)) == cudaSuccess, "cudaMalloc fields");
    CHECK(cudaMalloc(&phi_out, n * sizeof(float)) == cudaSuccess, "cudaMalloc phi");
    CHECK(cudaMemcpy(init, h, 3 * n * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess, "copy in");
    const double* d = (const double*)init;

    lbm_ctx* ctx = NULL;
    CHECK(lbm_init(&p, state, work, d, d + n, d + 2 * n, NULL, &ctx) == LBM_OK, lbm_last_error(NULL));
    double s0[LBM_NRED], s1[LBM_NRED];
    CHECK(lbm_reduce(ctx, s0) == LBM_OK, lbm_last_error(ctx));
    /* one step at a time so that the source budget can be summed step by step */
    double source = 0.0, s[LBM_NRED];
    for (int t = 0; t < 40; ++t) {
        CHECK(lbm_reduce(ctx, s) == LBM_OK, lbm_last_error(ctx));
        source += s[LBM_RED_S];
        CHECK(lbm_step(ctx, 1) == LBM_OK, lbm_last_error(ctx));
    }
    CHECK(lbm_reduce(ctx, s1) == LBM_OK, lbm_last_error(ctx));
    CHECK(lbm_time(ctx) == 40, "time level");

    void* dst[LBM_NFIELDS] = {0};
    dst[LBM_FIELD_PHI] = phi_out;
    CHECK(lbm_fields(ctx, dst) == LBM_OK, lbm_last_error(ctx));
    float* hp = (float*)malloc(n * sizeof(float));
    CHECK(hp != NULL, "host allocation");
    CHECK(cudaMemcpy(hp, phi_out, n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess, "copy out");
    float lo = 1e30f, hi = -1e30f;
    for (size_t i = 0; i < n; ++i) { lo = hp[i] < lo ? hp[i] : lo; hi = hp[i] > hi ? hp[i] : hi; }

    const double dA = fabs(s1[LBM_RED_C_A] - s0[LBM_RED_C_A]) / s0[LBM_RED_C_A];
    const double dB = fabs(s1[LBM_RED_C_B] - s0[LBM_RED_C_B]) / s0[LBM_RED_C_B];
    const double dP = fabs(s1[LBM_RED_P] - s0[LBM_RED_P]);
    const double dG = fabs(s1[LBM_RED_G] - (s0[LBM_RED_G] + source)) / s0[LBM_RED_G];
    CHECK(s1[LBM_RED_NONFINITE] == 0.0, "non-finite moments");
    CHECK(dA < 1e-6 && dB < 1e-6, "sum c drifted");
    CHECK(dP < 1e-6 * n * 1e-3, "sum p_h drifted");
    CHECK(dG < 1e-6, "sum g budget");
    CHECK(lo > -1e-3f && hi < 1.0f + 1e-3f, "phi out of [0, 1]");
    CHECK(s1[LBM_RED_UMAX] > 0.0 && s1[LBM_RED_UMAX] < 0.05, "max |u|");
    printf("c_abi_example ok: %s; rel drift c^A %.2e c^B %.2e, sum g budget %.2e, phi in [%.4f, %.4f], "
           "max|u| %.3e\n", lbm_build_info(), dA, dB, dG, lo, hi, s1[LBM_RED_UMAX]);
    lbm_destroy(ctx);
    cudaFree(state); cudaFree(work); cudaFree(init); cudaFree(phi_out);
    free(h); free(hp);
    return 0;
}
