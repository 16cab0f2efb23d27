// Kernels of the coupled step (§3), templated on storage type T, scalar lattice LAT,
// flow, and AA parity. Each translation unit lbm_step_<type>.cu instantiates them for
// one storage type through LBM_DEFINE_LAUNCHERS.
#pragma once

#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

constexpr int kBlockX = 128;

// Incoming populations of one node and their moments (steps a1-a3 of one node).
template <class T, int LAT, bool FLOW>
struct Node {
    using R = typename RealOf<T>::type;
    static constexpr int Q = Scalar<LAT>::Q;
    R g[Q], hA[Q], hB[Q];
    R f[FLOW ? 19 : 1];
    R phit, cA, cB, S;

    __device__ __forceinline__ void gather(const StateView& st, bool odd, int x, int y, int z,
                                           long long self, const DevParams& P) {
        const T* G = static_cast<const T*>(st.g);
        const T* HA = static_cast<const T*>(st.hA);
        const T* HB = static_cast<const T*>(st.hB);
        const float* rg = st.rest;
        const float* ra = st.rest ? st.rest + P.plane : nullptr;
        const float* rb = st.rest ? st.rest + 2 * P.plane : nullptr;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            Slot s = read_slot(odd, k, Scalar<LAT>::ex(k), Scalar<LAT>::ey(k), Scalar<LAT>::ez(k), x, y, z, self, P);
            g[k] = load_scalar<T, SET_G, LAT>(G, rg, k, s, P);
            hA[k] = load_scalar<T, SET_H, LAT>(HA, ra, k, s, P);
            hB[k] = load_scalar<T, SET_H, LAT>(HB, rb, k, s, P);
        }
        if constexpr (FLOW) {
            const T* F = static_cast<const T*>(st.f);
#pragma unroll
            for (int k = 0; k < 19; ++k) {
                Slot s = read_slot(odd, k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k), x, y, z, self, P);
                f[k] = Codec<T>::template load<SET_F>(F + (long long)s.slot * P.plane + s.node, D3Q19::w(k), P);
            }
        }
    }

    // Eq. 49 without the source, Eq. 52, Eq. 33 at phi~ and Eq. 35
    __device__ __forceinline__ void moments(const DevParams& P) {
        phit = R(0); cA = R(0); cB = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) { phit += g[k]; cA += hA[k]; cB += hB[k]; }
        R pt = interp_p(phit);
        S = source(phit, closure(cA, pt, 0, P), closure(cB, pt, 1, P), P);
    }
    __device__ __forceinline__ R phi() const { return phit + R(0.5) * S; }
};

// phi at x + e with periodic wrap and a mirror ghost across walls (zero normal gradient).
template <class R>
__device__ __forceinline__ R phi_at(const R* __restrict__ phi, int x, int y, int z, int dx, int dy, int dz,
                                    const DevParams& P) {
    int xx = x + dx, yy = y + dy, zz = z + dz;
    if (xx < 0 || xx >= P.nx) xx = P.wall_x ? x : (xx < 0 ? xx + P.nx : xx - P.nx);
    if (yy < 0) yy += P.ny; else if (yy >= P.ny) yy -= P.ny;
    if (zz < 0 || zz >= P.nz) zz = P.wall_z ? z : (zz < 0 ? zz + P.nz : zz - P.nz);
    return phi[node_of(xx, yy, zz, P)];
}

// Eqs. 42-45 regrouped over opposite pairs: grad = 3 sum_k w_k e_k phi(x+e_k),
// lap = 6 sum_k w_k (phi(x+e_k) - phi(x)), k = 1..18 of D3Q19.
template <class R>
__device__ __forceinline__ void stencil(const R* __restrict__ phi, int x, int y, int z, R phic,
                                        const DevParams& P, R& gx, R& gy, R& gz, R& lap) {
    gx = gy = gz = lap = R(0);
#pragma unroll
    for (int k = 1; k < 19; ++k) {
        R v = phi_at(phi, x, y, z, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k), P);
        R w = R(D3Q19::w(k));
        gx += w * R(D3Q19::ex(k)) * v;
        gy += w * R(D3Q19::ey(k)) * v;
        gz += w * R(D3Q19::ez(k)) * v;
        lap += w * (v - phic);
    }
    gx *= R(3); gy *= R(3); gz *= R(3); lap *= R(6);
}

// Total force (Eq. 34 + Boussinesq) and velocity (Eq. 41).
template <class R>
__device__ __forceinline__ void force_velocity(const R* f, R phi, R gx, R gy, R gz, R lap, const DevParams& P,
                                               R& Fx, R& Fy, R& Fz, R& ux, R& uy, R& uz) {
    R br = R(P.sw15) * (dwell_d(phi) * R(P.inv_W2) - lap);
    Fx = br * gx + phi * R(P.g[0]);
    Fy = br * gy + phi * R(P.g[1]);
    Fz = br * gz + phi * R(P.g[2]);
    R jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int k = 1; k < 19; ++k) {
        if (D3Q19::ex(k)) jx += R(D3Q19::ex(k)) * f[k];
        if (D3Q19::ey(k)) jy += R(D3Q19::ey(k)) * f[k];
        if (D3Q19::ez(k)) jz += R(D3Q19::ez(k)) * f[k];
    }
    ux = R(3) * jx + R(0.5) * Fx;
    uy = R(3) * jy + R(0.5) * Fy;
    uz = R(3) * jz + R(0.5) * Fz;
}

// ------------------------------------------------------------------------------------
// The fused step: gather (AA parity), moments, closure, source, [stencil, force, u],
// BGK collisions of f, g, h^A, h^B, scatter (AA parity, bounce-back at walls).
template <class T, int LAT, bool FLOW, bool ODD>
__global__ void __launch_bounds__(kBlockX)
step_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ phi_field) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    constexpr int Q = L::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long self = node_of(x, y, z, P);

    Node<T, LAT, FLOW> nd;
    nd.gather(st, ODD, x, y, z, self, P);
    nd.moments(P);
    const R S = nd.S;
    R phi;
    if constexpr (FLOW) phi = phi_field[self]; else phi = nd.phi();
    const R p = interp_p(phi);
    const R muA = closure(nd.cA, p, 0, P);
    const R muB = closure(nd.cB, p, 1, P);

    R ux = R(0), uy = R(0), uz = R(0);
    if constexpr (FLOW) {
        R gx, gy, gz, lap, Fx, Fy, Fz;
        stencil(phi_field, x, y, z, phi, P, gx, gy, gz, lap);
        force_velocity(nd.f, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
        // Eqs. 36-39: He-Shan-Doolen forcing, He-Luo equilibrium shifted by -F_k/2
        R ph = R(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) ph += nd.f[k];
        const R usq = ux * ux + uy * uy + uz * uz;
        const R omf = R(P.om_f);
        T* F = static_cast<T*>(st.f);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const R w = R(D3Q19::w(k));
            const R cu = R(D3Q19::ex(k)) * ux + R(D3Q19::ey(k)) * uy + R(D3Q19::ez(k)) * uz;
            const R gam = w * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
            const R Fk = gam * ((R(D3Q19::ex(k)) - ux) * Fx + (R(D3Q19::ey(k)) - uy) * Fy + (R(D3Q19::ez(k)) - uz) * Fz);
            const R feq = w * (ph + cu + R(1.5) * cu * cu - R(0.5) * usq) - R(0.5) * Fk;
            const R post = nd.f[k] - omf * (nd.f[k] - feq) + Fk;
            Slot s = write_slot(ODD, k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k), x, y, z, self, P);
            Codec<T>::template store<SET_F>(F + (long long)s.slot * P.plane + s.node, post, D3Q19::w(k), P);
        }
    }

    // Eqs. 46-48: g
    const R inv_cs2 = R(L::cs2() == 0.25 ? 4.0 : 3.0);
    const R omg = R(P.om_g);
    // Eqs. 50-51 with M^alpha(phi) of §2.3 and tau_h = M / c_s^2
    const R MA = R(P.M0[0]) * (R(1) - phi) + R(P.M1[0]) * phi;
    const R MB = R(P.M0[1]) * (R(1) - phi) + R(P.M1[1]) * phi;
    const R omA = R(1) / (MA * inv_cs2 + R(0.5));
    const R omB = R(1) / (MB * inv_cs2 + R(0.5));
    T* G = static_cast<T*>(st.g);
    T* HA = static_cast<T*>(st.hA);
    T* HB = static_cast<T*>(st.hB);
    float* rg = st.rest;
    float* ra = st.rest ? st.rest + P.plane : nullptr;
    float* rb = st.rest ? st.rest + 2 * P.plane : nullptr;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const R w = R(L::w(k));
        const R cu = R(L::ex(k)) * ux + R(L::ey(k)) * uy + R(L::ez(k)) * uz;
        const R geq = w * phi * (R(1) + inv_cs2 * cu) - R(0.5) * w * S;
        const R gpost = nd.g[k] - omg * (nd.g[k] - geq) + w * S;
        R heqA, heqB;
        if (k == 0) {
            heqA = nd.cA - (R(1) - w) * muA;
            heqB = nd.cB - (R(1) - w) * muB;
        } else {
            heqA = w * muA + w * nd.cA * inv_cs2 * cu;
            heqB = w * muB + w * nd.cB * inv_cs2 * cu;
        }
        const R hApost = nd.hA[k] - omA * (nd.hA[k] - heqA);
        const R hBpost = nd.hB[k] - omB * (nd.hB[k] - heqB);
        Slot s = write_slot(ODD, k, L::ex(k), L::ey(k), L::ez(k), x, y, z, self, P);
        store_scalar<T, SET_G, LAT>(G, rg, k, s, gpost, P);
        store_scalar<T, SET_H, LAT>(HA, ra, k, s, hApost, P);
        store_scalar<T, SET_H, LAT>(HB, rb, k, s, hBpost, P);
    }
}

// phi = sum g + S/2 of every node (Eq. 49), read by the capillary stencil of the flow step.
template <class T, int LAT, bool ODD>
__global__ void __launch_bounds__(kBlockX)
phi_kernel(const DevParams P, const StateView st, typename RealOf<T>::type* __restrict__ phi_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long self = node_of(x, y, z, P);
    Node<T, LAT, false> nd;
    nd.gather(st, ODD, x, y, z, self, P);
    nd.moments(P);
    phi_out[self] = nd.phi();
}

// Initial populations (time 0, even layout), computed in FP64 then stored.
template <class T, int LAT, bool FLOW>
__global__ void __launch_bounds__(kBlockX)
init_kernel(const DevParams P, const StateView st, const double* __restrict__ phi0,
            const double* __restrict__ cA0, const double* __restrict__ cB0) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long self = node_of(x, y, z, P);
    const double ph = phi0[self];
    const double cA = cA0[self], cB = cB0[self];
    const double pp = interp_p(ph);
    const double muA = closure(cA, pp, 0, P), muB = closure(cB, pp, 1, P);
    const double S0 = source(ph, muA, muB, P);
    T* G = static_cast<T*>(st.g);
    T* HA = static_cast<T*>(st.hA);
    T* HB = static_cast<T*>(st.hB);
    float* rg = st.rest;
    float* ra = st.rest ? st.rest + P.plane : nullptr;
    float* rb = st.rest ? st.rest + 2 * P.plane : nullptr;
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const double w = L::w(k);
        const Slot s{self, k};
        store_scalar<T, SET_G, LAT>(G, rg, k, s, R(w * ph - 0.5 * w * S0), P);          // Eq. 47, u = 0
        store_scalar<T, SET_H, LAT>(HA, ra, k, s, R(k == 0 ? cA - (1.0 - w) * muA : w * muA), P);  // Eq. 51
        store_scalar<T, SET_H, LAT>(HB, rb, k, s, R(k == 0 ? cB - (1.0 - w) * muB : w * muB), P);
    }
    if constexpr (FLOW) {
        double gx, gy, gz, lap;
        stencil(phi0, x, y, z, ph, P, gx, gy, gz, lap);
        const double br = P.sw15 * (dwell_d(ph) * P.inv_W2 - lap);
        const double Fx = br * gx + ph * P.g[0], Fy = br * gy + ph * P.g[1], Fz = br * gz + ph * P.g[2];
        T* F = static_cast<T*>(st.f);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const double w = D3Q19::w(k);
            const double Fk = w * (D3Q19::ex(k) * Fx + D3Q19::ey(k) * Fy + D3Q19::ez(k) * Fz);  // Eqs. 37-38, u = 0
            Codec<T>::template store<SET_F>(F + (long long)k * P.plane + self, R(-0.5 * Fk), w, P);  // Eq. 39
        }
    }
}

// Macroscopic fields of the current time level.
template <class T, int LAT, bool FLOW, bool ODD>
__global__ void __launch_bounds__(kBlockX)
fields_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ phi_field,
              FieldPtrs out) {
    using R = typename RealOf<T>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long self = node_of(x, y, z, P);
    Node<T, LAT, FLOW> nd;
    nd.gather(st, ODD, x, y, z, self, P);
    nd.moments(P);
    R phi;
    if constexpr (FLOW) phi = phi_field[self]; else phi = nd.phi();
    const R p = interp_p(phi);
    R vals[LBM_NFIELDS_DEV];
    vals[0] = phi;
    vals[1] = closure(nd.cA, p, 0, P);
    vals[2] = closure(nd.cB, p, 1, P);
    vals[3] = nd.cA;
    vals[4] = nd.cB;
    vals[5] = R(0); vals[6] = R(0); vals[7] = R(0); vals[8] = R(0);
    vals[9] = nd.S;
    if constexpr (FLOW) {
        R gx, gy, gz, lap, Fx, Fy, Fz;
        stencil(phi_field, x, y, z, phi, P, gx, gy, gz, lap);
        force_velocity(nd.f, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, vals[6], vals[7], vals[8]);
        R ph = R(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) ph += nd.f[k];
        vals[5] = ph;
    }
#pragma unroll
    for (int i = 0; i < LBM_NFIELDS_DEV; ++i)
        if (out.p[i]) static_cast<R*>(out.p[i])[self] = vals[i];
}

// FP64 block partials of the global diagnostics (grid-stride over nodes).
template <class T, int LAT, bool FLOW, bool ODD>
__global__ void __launch_bounds__(256)
reduce_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ phi_field,
              double* __restrict__ partials) {
    using R = typename RealOf<T>::type;
    double acc[LBM_NRED_DEV];
#pragma unroll
    for (int i = 0; i < LBM_NRED_DEV; ++i) acc[i] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < P.n; id += stride) {
        const int x = int(id % P.nx);
        const int y = int((id / P.nx) % P.ny);
        const int z = int(id / ((long long)P.nx * P.ny));
        Node<T, LAT, FLOW> nd;
        nd.gather(st, ODD, x, y, z, id, P);
        nd.moments(P);
        R phi;
        if constexpr (FLOW) phi = phi_field[id]; else phi = nd.phi();
        double umag = 0.0, ph = 0.0;
        if constexpr (FLOW) {
            R gx, gy, gz, lap, Fx, Fy, Fz, ux, uy, uz;
            stencil(phi_field, x, y, z, phi, P, gx, gy, gz, lap);
            force_velocity(nd.f, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
            umag = sqrt(double(ux) * ux + double(uy) * uy + double(uz) * uz);
            R s = R(0);
#pragma unroll
            for (int k = 0; k < 19; ++k) s += nd.f[k];
            ph = s;
        }
        const double vals[5] = {double(phi), double(nd.cA), double(nd.cB), ph, double(nd.S)};
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 5; ++i) { acc[i] += vals[i]; finite = finite && isfinite(vals[i]); }
        finite = finite && isfinite(umag) && isfinite(double(nd.phit));
        acc[5] = fmax(acc[5], isfinite(umag) ? umag : 0.0);
        acc[6] += double(nd.phit);
        acc[7] += finite ? 0.0 : 1.0;
    }
    // block reduction: warp shuffles, then one warp over the warp results
    __shared__ double sm[LBM_NRED_DEV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < LBM_NRED_DEV; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) {
            double u = __shfl_down_sync(0xffffffffu, v, o);
            v = (i == 5) ? fmax(v, u) : v + u;
        }
        if (lane == 0) sm[i][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int i = 0; i < LBM_NRED_DEV; ++i) {
            double v = lane < nw ? sm[i][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                double u = __shfl_down_sync(0xffffffffu, v, o);
                v = (i == 5) ? fmax(v, u) : v + u;
            }
            if (lane == 0) partials[(long long)blockIdx.x * LBM_NRED_DEV + i] = v;
        }
    }
}

// ------------------------------------------------------------------------------------
// Host launchers for one storage type.
inline dim3 node_grid(const DevParams& P, int& bx) {
    bx = P.nx >= kBlockX ? kBlockX : ((P.nx + 31) / 32) * 32;
    return dim3((P.nx + bx - 1) / bx, P.ny, P.nz);
}

template <class T>
struct Launchers {
    using R = typename RealOf<T>::type;

    template <int LAT, bool FLOW>
    static void init(const DevParams& P, const StateView& st, const double* phi0, const double* cA0,
                     const double* cB0, cudaStream_t s) {
        int bx; dim3 grid = node_grid(P, bx);
        init_kernel<T, LAT, FLOW><<<grid, bx, 0, s>>>(P, st, phi0, cA0, cB0);
    }
    template <int LAT>
    static void phi(const DevParams& P, const StateView& st, bool odd, void* phi_work, cudaStream_t s) {
        int bx; dim3 grid = node_grid(P, bx);
        R* ph = static_cast<R*>(phi_work);
        if (odd) phi_kernel<T, LAT, true><<<grid, bx, 0, s>>>(P, st, ph);
        else phi_kernel<T, LAT, false><<<grid, bx, 0, s>>>(P, st, ph);
    }
    // the fused step kernel; with flow, the phi pass of the same step must precede it
    template <int LAT, bool FLOW>
    static void step(const DevParams& P, const StateView& st, bool odd, void* phi_work, cudaStream_t s) {
        int bx; dim3 grid = node_grid(P, bx);
        R* phi = static_cast<R*>(phi_work);
        if (odd) step_kernel<T, LAT, FLOW, true><<<grid, bx, 0, s>>>(P, st, phi);
        else step_kernel<T, LAT, FLOW, false><<<grid, bx, 0, s>>>(P, st, phi);
    }
    template <int LAT, bool FLOW>
    static void fields(const DevParams& P, const StateView& st, bool odd, void* phi_work, FieldPtrs out,
                       cudaStream_t s) {
        int bx; dim3 grid = node_grid(P, bx);
        R* phi = static_cast<R*>(phi_work);
        if constexpr (FLOW) {
            if (odd) phi_kernel<T, LAT, true><<<grid, bx, 0, s>>>(P, st, phi);
            else phi_kernel<T, LAT, false><<<grid, bx, 0, s>>>(P, st, phi);
        }
        if (odd) fields_kernel<T, LAT, FLOW, true><<<grid, bx, 0, s>>>(P, st, phi, out);
        else fields_kernel<T, LAT, FLOW, false><<<grid, bx, 0, s>>>(P, st, phi, out);
    }
    template <int LAT, bool FLOW>
    static void reduce(const DevParams& P, const StateView& st, bool odd, void* phi_work, double* partials,
                       int nblocks, cudaStream_t s) {
        R* phi = static_cast<R*>(phi_work);
        if constexpr (FLOW) {
            int bx; dim3 grid = node_grid(P, bx);
            if (odd) phi_kernel<T, LAT, true><<<grid, bx, 0, s>>>(P, st, phi);
            else phi_kernel<T, LAT, false><<<grid, bx, 0, s>>>(P, st, phi);
        }
        if (odd) reduce_kernel<T, LAT, FLOW, true><<<nblocks, 256, 0, s>>>(P, st, phi, partials);
        else reduce_kernel<T, LAT, FLOW, false><<<nblocks, 256, 0, s>>>(P, st, phi, partials);
    }
};

// Dispatch over (lattice, flow) for one storage type.
#define LBM_DEFINE_LAUNCHERS(T, SUFFIX)                                                              \
    void launch_init_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow,           \
                              const double* a, const double* b, const double* c, cudaStream_t s) {   \
        if (lat == LAT_D2Q5) Launchers<T>::init<LAT_D2Q5, false>(P, st, a, b, c, s);                  \
        else if (flow) Launchers<T>::init<LAT_D3Q7, true>(P, st, a, b, c, s);                         \
        else Launchers<T>::init<LAT_D3Q7, false>(P, st, a, b, c, s);                                  \
    }                                                                                                \
    void launch_phi_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool odd, void* phi,      \
                             cudaStream_t s) {                                                       \
        if (lat == LAT_D2Q5) Launchers<T>::phi<LAT_D2Q5>(P, st, odd, phi, s);                         \
        else Launchers<T>::phi<LAT_D3Q7>(P, st, odd, phi, s);                                         \
    }                                                                                                \
    void launch_step_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, bool odd,  \
                              void* phi, cudaStream_t s) {                                           \
        if (lat == LAT_D2Q5) Launchers<T>::step<LAT_D2Q5, false>(P, st, odd, phi, s);                 \
        else if (flow) Launchers<T>::step<LAT_D3Q7, true>(P, st, odd, phi, s);                        \
        else Launchers<T>::step<LAT_D3Q7, false>(P, st, odd, phi, s);                                 \
    }                                                                                                \
    void launch_fields_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, bool odd,\
                                void* phi, FieldPtrs out, cudaStream_t s) {                          \
        if (lat == LAT_D2Q5) Launchers<T>::fields<LAT_D2Q5, false>(P, st, odd, phi, out, s);          \
        else if (flow) Launchers<T>::fields<LAT_D3Q7, true>(P, st, odd, phi, out, s);                 \
        else Launchers<T>::fields<LAT_D3Q7, false>(P, st, odd, phi, out, s);                          \
    }                                                                                                \
    void launch_reduce_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, bool odd,\
                                void* phi, double* partials, int nblocks, cudaStream_t s) {          \
        if (lat == LAT_D2Q5) Launchers<T>::reduce<LAT_D2Q5, false>(P, st, odd, phi, partials, nblocks, s); \
        else if (flow) Launchers<T>::reduce<LAT_D3Q7, true>(P, st, odd, phi, partials, nblocks, s);   \
        else Launchers<T>::reduce<LAT_D3Q7, false>(P, st, odd, phi, partials, nblocks, s);            \
    }

}  // namespace lbm
