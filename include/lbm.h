/*
 * C-ABI of the GB300 (sm_103a) grand-potential phase-field lattice Boltzmann step.
 *
 * The method (Verdier, Cartalade, Plapp, "Grand-potential phase field simulations
 * of droplet growth and sedimentation in a two-phase ternary fluid") couples, on
 * one lattice, four lattice Boltzmann equations:
 *   g     - the Allen-Cahn phase field phi with its source S_phi   (§3.2, Eqs. 46-49, 35)
 *   h^A,B - the compositions c^A, c^B; mu from the closure Eq. 33  (§3.3, Eqs. 50-52)
 *   f     - incompressible flow with capillary + buoyancy forcing  (§3.1, Eqs. 36-45, 34)
 * g, h^A, h^B use D2Q5 or D2Q9 (2D), D3Q7 or D3Q19 (3D) with BGK collisions; f uses
 * D3Q19 with a BGK, TRT or MRT collision.
 * One call of lbm_step advances every population set by one fused collide-and-stream
 * pass over HBM: in-place AA-pattern streaming without flow; with flow, by default, a
 * two-buffer pull step that computes the capillary stencil's phi on the fly.
 *
 * Memory: every device buffer is allocated and owned by the caller (for instance a
 * torch tensor); the library never allocates or frees device memory. The context is
 * a small host object. All work is queued on the caller's CUDA stream; only
 * lbm_reduce synchronises that stream.
 *
 * Errors: every entry point returns an lbm_status; nothing aborts, traps or exits.
 * lbm_last_error gives a message for the last failure on a context.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument: sizes, enum values, null pointers, alignment */
    LBM_ERR_CUDA = -2,      /* a CUDA call failed; lbm_last_error has the CUDA message */
    LBM_ERR_UNSTABLE = -3,  /* lbm_reduce found a non-finite value in the state */
    LBM_ERR_STATE = -4      /* call out of order (e.g. adjoint on a flow lattice) */
} lbm_status;

/* Lattice of the phi, c^A and c^B populations (the flow always uses D3Q19). LBM_D2Q5 and
 * LBM_D3Q7 are the minimal advection-diffusion sets; LBM_D3Q19 (3D) and LBM_D2Q9 (2D) are
 * the paper's choices (§3). The 2D lattices need nz = 1 and carry no flow. With flow and two
 * state copies, LBM_D3Q7 runs the fused z-marching kernel; LBM_D3Q19 runs a phi pass and a
 * per-node pull step instead. */
typedef enum { LBM_D2Q5 = 0, LBM_D3Q7 = 1, LBM_D3Q19 = 2, LBM_D2Q9 = 3 } lbm_lattice;

/* Storage type of the populations. Arithmetic is FP64 for LBM_F64 and FP32 otherwise.
 * LBM_F16 / LBM_BF16 store every moving population (k > 0) in 16 bits as its value per unit
 * weight: x_k = g_k / w_k - 1/2, x_k = h_k / w_k, and for f the deviation from the rest
 * population of the node that stored it, x_k = f_k / w_k - f_0 / w_0 (f_0 ~ w_0 p_h, so the
 * pressure is not rounded). The rest populations g_0, h^A_0, h^B_0, f_0 stay FP32 (in place,
 * f_0 alternates between two planes by the parity of the time level).
 *   LBM_F16: g in 16-bit fixed point over [-1, 1) (step 2^-15, saturating: a stable run
 *            stays far inside); f as IEEE FP16 of 1024 x_k, h as IEEE FP16 of 64 x_k.
 *   LBM_BF16: every x_k as BF16 (8-bit significand).
 * Every step sets the rest populations of g and h to their set's conserved total at the node
 * (phi~ + S, c - c_0^eq) minus the moving populations as stored, so phi, c^A and c^B are
 * carried to FP32 accuracy and 16-bit rounding cannot act as a source of composition; the
 * f_0 of a node is its collided value, so sum p_h carries the 16-bit rounding of the moving
 * f (the pressure is defined up to a constant in the incompressible limit).
 * In every storage type the rest populations h^alpha_0 are kept shifted by the constant
 * c_0^{alpha,eq} (h_0 - c_0^eq), so that the sum of the h populations is c - c_0^eq and
 * mu (Eq. 33) does not inherit the rounding of c itself. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 } lbm_storage;

/* Flow collision operators. LBM_BGK is the paper's single-rate operator (Eq. 36). LBM_TRT and
 * LBM_MRT are the two- and multiple-relaxation-time operators the paper names as
 * alternatives (§3). TRT: the parts of f - f^eq even and odd under k -> opp(k) relax at
 * omega+ and omega-. MRT: the moments of f - f^eq on d'Humieres' orthogonal D3Q19 basis relax
 * at their own rates (shear moments at omega of Eq. 36). In both, f^eq keeps the -F_k/2 shift
 * of Eq. 39 and F_k is added as in Eq. 36. */
typedef enum { LBM_BGK = 0, LBM_TRT = 1, LBM_MRT = 2 } lbm_collision;

/* Model parameters in lattice units (dx = dt = 1, rho_0 = 1), named as in the paper. */
typedef struct lbm_params {
    int32_t nx, ny, nz;      /* lattice extents; nz = 1 with the 2D lattices (LBM_D2Q5, LBM_D2Q9) */
    int32_t lattice;         /* lbm_lattice of g, h^A, h^B */
    int32_t flow;            /* 1: D3Q19 flow populations, capillary (Eq. 34) + buoyancy forcing */
    int32_t storage;         /* lbm_storage */
    int32_t wall_x;          /* 1: half-way bounce-back planes at x = -1/2 and nx - 1/2 */
    int32_t wall_z;          /* 1: half-way bounce-back planes at z = -1/2 and nz - 1/2 */
    int32_t source_off;      /* 1: S_phi = 0 (pure advection-diffusion of phi; test switch) */
    int32_t inplace;         /* flow only. 0: two state copies, one fused kernel per step (the
                              * capillary stencil's phi is computed on the fly in shared memory);
                              * 1: one in-place AA-pattern copy (half the memory) plus a phi pass.
                              * Without flow the state is always one in-place AA-pattern copy. */
    double W;                /* interface width (Eq. 14) */
    double lambda;           /* coupling constant lambda = K / H (§2.2) */
    double M_phi;            /* scaled phase-field mobility, M_phi = W^2 / tau_phi */
    double c_eq[2][2];       /* c_eq[pi][alpha]: equilibrium composition of phase pi, component alpha */
    double M[2][2];          /* M[pi][alpha]: mobility of component alpha in phase pi (§2.3) */
    double nu;               /* kinematic viscosity, tau_f = nu / c_s^2 (Eq. 36) */
    double sigma;            /* surface tension in Eq. 34 */
    double g[3];             /* buoyancy per unit phi: F_g = phi * g (§2.5, Delta rho g / rho_0) */
    double f_scale;          /* reserved: 0 or 1024 (the 16-bit formats have fixed scales) */
    int32_t collision;       /* flow collision, lbm_collision: LBM_BGK (Eq. 36), LBM_TRT or LBM_MRT */
    double trt_magic;        /* LBM_TRT: Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) > 0, where omega+
                              * is the BGK rate of Eq. 36 (it sets nu); 0 selects 3/16 */
    double mrt_rates[5];     /* LBM_MRT: rates in (0, 2) of the energy, energy-square, energy-flux,
                              * pi and m moments; 0 selects 1.19, 1.4, 1.2, 1.4, 1.98 */
} lbm_params;

/* Indices of lbm_fields outputs. */
enum {
    LBM_FIELD_PHI = 0, LBM_FIELD_MU_A, LBM_FIELD_MU_B, LBM_FIELD_C_A, LBM_FIELD_C_B,
    LBM_FIELD_P, LBM_FIELD_UX, LBM_FIELD_UY, LBM_FIELD_UZ, LBM_FIELD_S,
    LBM_NFIELDS
};

/* Indices of lbm_reduce outputs. */
enum {
    LBM_RED_PHI = 0,     /* sum phi (Eq. 49) */
    LBM_RED_C_A,         /* sum c^A (Eq. 52), invariant */
    LBM_RED_C_B,         /* sum c^B, invariant */
    LBM_RED_P,           /* sum p_h (Eq. 40), invariant */
    LBM_RED_S,           /* sum S_phi: the next step changes sum g by exactly this */
    LBM_RED_UMAX,        /* max |u| (Eq. 41) */
    LBM_RED_G,           /* sum of all g populations (= sum phi - sum S / 2) */
    LBM_RED_NONFINITE,   /* number of nodes with a non-finite moment */
    LBM_RED_INTERFACE,   /* sum (4/W) phi (1 - phi): interface length (2D) or area (3D); Eq. 67 gives
                          * the mean droplet radius <R> = this / (2 pi N) in 2D */
    LBM_RED_EULER,       /* Euler characteristic of {phi >= 1/2} taken as the union of closed
                          * unit squares (2D: 8-connected droplets, Gray's 2x2 bit quads) or
                          * cubes (3D: 26-connected, vertices - edges + faces - cubes of that
                          * union, each node owning the cells at its low corner); outside an
                          * x or z wall is empty. It is the droplet count N when no droplet
                          * has a hole or a handle (§4.2.2 measures N this way). A 3D lattice
                          * with nz == 1 and no z walls is a slab closed on itself: 0 */
    LBM_NRED
};

typedef struct lbm_ctx lbm_ctx;

/* Bytes of the population state for these parameters (256-byte aligned planes). */
size_t lbm_state_bytes(const lbm_params* p);

/* Bytes of scratch the step needs beside the state: the phi field (read by the capillary
 * stencil with flow, and by the droplet count of lbm_reduce on the 2D lattices), one bit
 * per node of phi >= 1/2 (the droplet count of lbm_reduce on the 3D lattices) and the
 * block partials of lbm_reduce. */
size_t lbm_work_bytes(const lbm_params* p);

/* Validate p, bind the caller's device buffers and CUDA stream (cudaStream_t passed as
 * void*, NULL = legacy default stream), and write the initial populations at rest
 * (§4.2.1): g = w phi0 - w S0/2, h = h^eq(c0, mu0) with mu0 from Eq. 33, f = f^eq at
 * p_h = 0, u = 0 shifted by the initial forcing. d_phi0, d_cA0, d_cB0 are FP64 device
 * arrays of nx*ny*nz values, x fastest; they are read during the call's kernel and may
 * be freed once the stream has passed it. d_state (lbm_state_bytes) and d_work
 * (lbm_work_bytes) must be 256-byte aligned and stay valid until lbm_destroy.
 * On success *out receives a new context (time 0). */
lbm_status lbm_init(const lbm_params* p, void* d_state, void* d_work,
                    const double* d_phi0, const double* d_cA0, const double* d_cB0,
                    void* stream, lbm_ctx** out);

/* Bind buffers whose state was written earlier (checkpoint/resume; the paper describes
 * none): d_state must hold a state produced by this library for the same parameters at
 * time t. No kernel runs. */
lbm_status lbm_attach(const lbm_params* p, void* d_state, void* d_work, int64_t t,
                      void* stream, lbm_ctx** out);

/* Advance nsteps >= 0 coupled time steps (§3): one fused collide-and-stream kernel per
 * step; with flow, the in-place layout and the LBM_D3Q19 scalar lattice add a phi pass for
 * the capillary stencil (lbm_kernels_per_step). Asynchronous. */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Advance nsteps coupled time steps by replaying a CUDA graph of two steps (captured on the
 * first call from an even time level, after one plain pair of steps; kept until
 * lbm_destroy): the same kernels and results as lbm_step, bit for bit, with one launch per
 * two steps, for lattices small enough that launch overhead shows. The context's stream must
 * be one the caller created (the legacy and per-thread default streams cannot be captured:
 * LBM_ERR_ARG). The replayed graph holds the buffers bound at lbm_init/lbm_attach; steps run
 * this way are not recorded by lbm_profile_begin. No counterpart in the paper. */
lbm_status lbm_step_graph(lbm_ctx* ctx, int nsteps);

/* Current time level (number of steps since lbm_init, or t of lbm_attach); -1 for NULL. */
int64_t lbm_time(const lbm_ctx* ctx);

/* Macroscopic fields of the current time level into caller device buffers:
 * dst[LBM_NFIELDS] pointers, NULL for fields not wanted; each holds nx*ny*nz values,
 * x fastest, in double for LBM_F64 and float otherwise. phi = sum g + S/2 (Eq. 49),
 * mu by Eq. 33, c by Eq. 52, p by Eq. 40, u by Eq. 41 (0 without flow). Asynchronous. */
lbm_status lbm_fields(lbm_ctx* ctx, void* const* dst);

/* FP64 global diagnostics of the current time level into host memory out[LBM_NRED]: the
 * sums of Eqs. 40, 49, 52, max |u| (§4.2.4), the interface measure of Eq. 67 and the droplet
 * count of §4.2.2 (LBM_RED_*). Per-node values are formed in the storage's arithmetic type
 * and summed with FP64 accuracy (float-float FP32 pairs per thread for FP32 arithmetic).
 * Synchronises the stream. Returns LBM_ERR_UNSTABLE if a moment is not finite. */
lbm_status lbm_reduce(lbm_ctx* ctx, double* out);

/* Kernel timing on the context's stream (no counterpart in the paper).
 * lbm_profile_begin(ctx, max_steps) creates
 * 3 * max_steps CUDA events (host-side driver objects, no device memory); each of the
 * next max_steps steps records one event before, between and after its kernels.
 * lbm_profile_end synchronises the stream and writes out[0] = total ms of the phi
 * passes, out[1] = total ms of the fused step kernels, out[2] = steps timed, then
 * destroys the events. */
lbm_status lbm_profile_begin(lbm_ctx* ctx, int max_steps);
lbm_status lbm_profile_end(lbm_ctx* ctx, double* out);

/* Number of kernels one lbm_step(ctx, 1) launches: 2 with flow unless the state has two
 * copies and the scalar lattice is LBM_D3Q7 (the fused kernel), else 1; 0 for NULL. */
int lbm_kernels_per_step(const lbm_ctx* ctx);

/* One step (§3) out of place, without a context: d_src holds one state copy at time t (the
 * layout lbm_init writes: lbm_copy_bytes bytes), d_dst receives time t + 1 in the same
 * layout; d_src is not modified. d_work as for lbm_init (used by in-place flow). The
 * adjoint's recompute pass uses it to rebuild the states of a segment from a checkpoint. */
lbm_status lbm_step_buffers(const lbm_params* p, const void* d_src, void* d_dst, int64_t t,
                            void* d_work, void* stream);

/* Bytes of one state copy (lbm_state_bytes is one or two copies). */
size_t lbm_copy_bytes(const lbm_params* p);

/* ---- Discrete adjoint of the coupled step without flow (storage LBM_F32 or LBM_F64) ----
 * The method's reverse mode: with Lambda_t = dL/dP_t the adjoint of the incoming
 * populations at time t (canonical layout: 3*Q planes ordered g, h^A, h^B, each plane
 * population k, element = node, in the arithmetic type), one reverse step is
 * Lambda_t = J_C(P_t)^T S^T Lambda_{t+1}, the transpose of the local BGK collision
 * (Eqs. 20, 33, 35, 46-51) after the reverse of the streaming; the gradient with respect to
 * the mobilities M[pi][alpha] and M_phi accumulates in FP64 in d_adj_work. Flow is not
 * supported (LBM_ERR_STATE). Everything is asynchronous on ``stream`` except
 * lbm_adjoint_theta. These calls allocate nothing. */
size_t lbm_adjoint_bytes(const lbm_params* p);       /* one Lambda field */
size_t lbm_adjoint_work_bytes(const lbm_params* p);  /* FP64 gradient partials */

/* Zero the gradient partials. */
lbm_status lbm_adjoint_reset(const lbm_params* p, void* d_adj_work, void* stream);

/* Lambda_T from the adjoint of the fields at time T: d_phib, d_muAb, d_muBb hold
 * dL/dphi, dL/dmu^A, dL/dmu^B per node (arithmetic type; NULL = zero); d_state is the state
 * copy at time t (in-place layout). Adds the M_phi part of the seed to the partials. */
lbm_status lbm_adjoint_seed(const lbm_params* p, const void* d_state, int64_t t, const void* d_phib,
                            const void* d_muAb, const void* d_muBb, void* d_lam, void* d_adj_work,
                            void* stream);

/* Lambda_t (d_lam) from Lambda_{t+1} (d_lam_next) at the state copy of time t. */
lbm_status lbm_adjoint_step(const lbm_params* p, const void* d_state, int64_t t, const void* d_lam_next,
                            void* d_lam, void* d_adj_work, void* stream);

/* One checkpoint segment of the reverse sweep in a single call: the states t0+1 .. t0+n-1
 * are recomputed out of place from the checkpoint in copy 0 of d_ring (n state copies,
 * lbm_copy_bytes apart) into copies 1 .. n-1, then the n reverse steps t0+n-1 .. t0 run from
 * Lambda_{t0+n} in d_lam, alternating with d_lam_tmp. *which receives 0 when Lambda_{t0}
 * ends in d_lam and 1 when it ends in d_lam_tmp. d_work as for lbm_init. */
lbm_status lbm_adjoint_segment(const lbm_params* p, void* d_ring, int64_t t0, int n, void* d_lam,
                               void* d_lam_tmp, void* d_adj_work, void* d_work, void* stream, int* which);

/* dL/dphi_0 (FP64, per node) from Lambda_0 through the initial populations of lbm_init;
 * adds the M_phi part of the initial source to the partials. */
lbm_status lbm_adjoint_init(const lbm_params* p, const double* d_phi0, const double* d_cA0,
                            const double* d_cB0, const void* d_lam0, double* d_phi0b, void* d_adj_work,
                            void* stream);

/* Sum the partials: out[0..4] = dL/dM[0][A], dL/dM[0][B], dL/dM[1][A], dL/dM[1][B], dL/dM_phi.
 * Synchronises the stream. */
lbm_status lbm_adjoint_theta(const lbm_params* p, void* d_adj_work, double* out, void* stream);

/* Mean droplet radius from the sums of lbm_reduce (or lbm_reduce_static): with A the
 * interface measure (LBM_RED_INTERFACE, Eq. 67's sum of (4/W) phi (1 - phi)) and N the
 * droplet count (LBM_RED_EULER), <R> = A / (2 pi N) on 2D lattices (Eq. 67) and
 * sqrt(A / (4 pi N)) on 3D lattices (the sum of the sphere areas). NaN when N <= 0 or an
 * argument is NULL. Host arithmetic only. */
double lbm_mean_radius(const lbm_params* p, const double* sums);

/* ------------------------------------------------------------------------------------
 * Slabs: a 3D lattice decomposed along z, the paper's domain decomposition for its
 * multi-GPU runs (§3; §4.2.4 ran 2048 x 512 x 512 on 64 GPUs). A slab owns the planes
 * [z0, z0 + nzl) of the lattice p describes and keeps one ghost plane on each side that has
 * a neighbour (another slab, or, where z is periodic, the slab across the periodic end; a
 * single slab covering a periodic lattice is its own neighbour). Slabs always use the
 * two-buffer layout (p->inplace must be 0); with flow and D3Q7 the step is the fused kernel.
 * The arithmetic per node is that of the undivided lattice, so a decomposed run equals it
 * bit for bit once the halos are exchanged as below.
 *
 * One step of the decomposed lattice, for every slab:
 *   1. lbm_step(ctx, 1) (a slab advances one step per call; larger counts are refused);
 *   2. populations: lbm_slab_pack(ctx, 0, m0) and lbm_slab_pack(ctx, 1, m1) write the
 *      populations that leave through the lower and upper face (5 flow and 1 or 5 per
 *      scalar set per face node; with 16-bit storage and flow also the FP32 f_0 of the edge
 *      plane, the reference of those f); the lower neighbour unpacks m0 at its side 1
 *      (lbm_slab_unpack(nbr, 1, m0)), the upper one m1 at its side 0;
 *   3. phi (flow only): after step 2, lbm_slab_phi_pack(ctx, side, buf) writes phi of the
 *      lowest (side 0) or highest (side 1) own plane; the neighbour on that side stores it
 *      with lbm_slab_phi_unpack at its opposite side. The capillary stencil of the edge
 *      planes reads it at the next step.
 * After lbm_slab_init only step 3 is needed before the first step (init places the ghost
 * populations itself). Messages are device buffers of lbm_slab_halo_bytes and
 * lbm_slab_phi_bytes; how they travel (a device copy, NCCL send/recv) is the caller's. */

/* Planes of a slab's own lattice (nzl plus its ghost planes); 0 for invalid arguments. The
 * initial fields of lbm_slab_init and the outputs of lbm_fields on a slab have this many z
 * planes: the global planes z0 - 1 .. z0 + nzl (wrapped at periodic ends; a plane beyond a
 * wall is not included). */
int32_t lbm_slab_planes(const lbm_params* p, int32_t z0, int32_t nzl);

/* Bytes of a slab's state (two copies of its own lattice) and work buffers; 0 for invalid
 * arguments. */
size_t lbm_slab_state_bytes(const lbm_params* p, int32_t z0, int32_t nzl);
size_t lbm_slab_work_bytes(const lbm_params* p, int32_t z0, int32_t nzl);

/* Initialise the slab [z0, z0 + nzl) of lattice p from FP64 fields over its lbm_slab_planes
 * planes (nx-fastest, the ghost planes included: the initial capillary stencil reads them).
 * Buffers as for lbm_init. On a slab context lbm_step takes at most one step per call,
 * lbm_step_graph and the adjoint are refused, lbm_fields writes the own planes of arrays
 * shaped like the initial fields, and lbm_reduce sums the own planes (its droplet count,
 * which needs the whole lattice, is 0). */
lbm_status lbm_slab_init(const lbm_params* p, int32_t z0, int32_t nzl, void* d_state, void* d_work,
                         const double* d_phi0, const double* d_cA0, const double* d_cB0, void* stream,
                         lbm_ctx** out);

/* Ghost planes of a slab context: bit 0 set when a neighbour lies below, bit 1 above; -1 if
 * ctx is not a slab. */
int32_t lbm_slab_ghosts(const lbm_ctx* ctx);

/* Size of one population message (both faces have the same) and of one phi message; 0 if
 * ctx is not a slab. */
size_t lbm_slab_halo_bytes(const lbm_ctx* ctx);
size_t lbm_slab_phi_bytes(const lbm_ctx* ctx);

/* Step 2 of the exchange: pack the populations leaving through face side (0 lower, 1 upper)
 * at the current time level into d_msg; unpack a neighbour's message into the ghost plane
 * on side (0: the message of the lower neighbour's upper face). Asynchronous on the
 * context's stream (device-to-device copies). LBM_ERR_STATE when the side has no
 * neighbour (a wall) or ctx is not a slab. */
lbm_status lbm_slab_pack(lbm_ctx* ctx, int32_t side, void* d_msg);
lbm_status lbm_slab_unpack(lbm_ctx* ctx, int32_t side, const void* d_msg);

/* Step 3: phi (Eq. 49, storage's arithmetic type) of the edge plane on side at the current
 * time level into d_phi (nx * ny values, x fastest; needs the ghost populations of step 2);
 * store a neighbour's edge-plane phi as the ghost phi on side. */
lbm_status lbm_slab_phi_pack(lbm_ctx* ctx, int32_t side, void* d_phi);
lbm_status lbm_slab_phi_unpack(lbm_ctx* ctx, int32_t side, const void* d_phi);

/* Allocation-free FP64 diagnostics. The paper has no counterpart: this is for callers that
 * cannot allocate device memory at the time they need the sums (for example a host
 * application that hands this library its state buffer but owns every allocation, or a
 * real-time loop where allocation is forbidden after start-up). Same results as
 * lbm_reduce for the state copy d_state holds at time t (the buffer lbm_init was given),
 * but the reduction's scratch (block partials and results; for flow or 2D lattices the phi
 * field, 4 bytes per node, 8 with LBM_F64; for 3D lattices one bit per node) lives in a
 * file-scope device array of 4 MiB that every GPU loading this library holds until the
 * process exits. After the 97 KB of partials the array holds the phi field of about
 * 1.02 million nodes (FP32 and 16-bit storage) or 0.51 million (LBM_F64), and the bit field
 * of about 33.5 million nodes (3D lattices without flow); larger lattices are rejected with
 * LBM_ERR_ARG before any launch. The call allocates nothing. d_state and the stream must
 * belong to the current device (LBM_ERR_ARG otherwise): the array's address is looked up,
 * with cudaGetSymbolAddress, for the current device on every call, so the very first call
 * on a device also loads the library's module there. Every call synchronises the stream and
 * copies the sums to the host, so it cannot be made while its stream is being captured into
 * a graph. Every call shares the array and leaves its contents behind; the kernels
 * overwrite all of it that they read, so nothing needs clearing, but calls that overlap on
 * the GPU (other streams, other host threads) race on it. */
lbm_status lbm_reduce_static(const lbm_params* p, const void* d_state, int64_t t, double* out, void* stream);

/* Release the context (host memory only; device buffers remain the caller's). */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Message of the last error on ctx (or of the last failed lbm_init/lbm_attach when
 * ctx is NULL). Never NULL. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Build and device information, for diagnostics: "sm_103a ..." */
const char* lbm_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
