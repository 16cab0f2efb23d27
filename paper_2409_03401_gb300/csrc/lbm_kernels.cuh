// Kernels of the coupled step (§3), templated on storage type T, scalar lattice LAT, flow,
// and streaming mode. Each translation unit lbm_step_<type>.cu instantiates them for one
// storage type through LBM_DEFINE_LAUNCHERS.
//
// Streaming modes:
//   AA_EVEN / AA_ODD - one in-place buffer (AA pattern): even steps read and write the
//                      node's own slots; odd steps read and write the neighbours' slots.
//   PULL             - two buffers: each step gathers incoming populations from the
//                      source buffer, which holds post-collision values at the node that
//                      produced them, and stores its own post-collision values locally
//                      (aligned, coalesced) in the destination buffer.
#pragma once

#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

constexpr int kBlockX = 128;
enum { AA_EVEN = 0, AA_ODD = 1, PULL = 2 };

// Wrapped neighbour coordinates of one node, computed once per thread. c[a][1 + d] is the
// coordinate x_a + d along axis a (d = -1, 0, 1) after the periodic wrap, or -1 where
// x_a + d lies beyond a wall.
struct Nbr {
    int c[3][3];
    int row[3][3];  // (z' ny + y') nx for z' = c[2][iz] (own plane beyond a wall), y' = c[1][iy]
    __device__ __forceinline__ void init(int x, int y, int z, const DevParams& P) {
        const int n[3] = {P.nx, P.ny, P.nz};
        const int w[3] = {P.wall_x, 0, P.wall_z};
        const int v[3] = {x, y, z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int d = -1; d <= 1; ++d) {
                int q = v[a] + d;
                if (q < 0) q = w[a] ? -1 : q + n[a];
                else if (q >= n[a]) q = w[a] ? -1 : q - n[a];
                c[a][d + 1] = q;
            }
        }
#pragma unroll
        for (int iz = 0; iz < 3; ++iz)
#pragma unroll
            for (int iy = 0; iy < 3; ++iy)
                row[iz][iy] = ((c[2][iz] < 0 ? z : c[2][iz]) * P.ny + c[1][iy]) * P.nx;
    }
    // node x + (dx, dy, dz); false (and the node itself) when that lies beyond a wall
    __device__ __forceinline__ bool at(int dx, int dy, int dz, int self, int& out) const {
        const int xx = c[0][dx + 1], zz = c[2][dz + 1];
        if (xx < 0 || zz < 0) { out = self; return false; }
        out = row[dz + 1][dy + 1] + xx;
        return true;
    }
};

// Where population k of this node is read from / written to, for each streaming mode.
// Across a wall both fall back to the node itself with k and opp(k) exchanged (half-way
// bounce-back).
template <int MODE>
__device__ __forceinline__ Slot src_slot(int k, int ex, int ey, int ez, const Nbr& nb, int self) {
    if (MODE == AA_EVEN || k == 0) return {self, k};
    int q;
    const bool in = nb.at(-ex, -ey, -ez, self, q);
    if (MODE == AA_ODD) return in ? Slot{q, opp(k)} : Slot{self, k};
    return in ? Slot{q, k} : Slot{self, opp(k)};
}
template <int MODE>
__device__ __forceinline__ Slot dst_slot(int k, int ex, int ey, int ez, const Nbr& nb, int self) {
    if (k == 0 || MODE == PULL) return {self, k};
    if (MODE == AA_EVEN) return {self, opp(k)};
    int q;
    return nb.at(ex, ey, ez, self, q) ? Slot{q, k} : Slot{self, opp(k)};
}

// Addressing of one node's populations through its wrapped neighbour table (branch-free
// selects, so warps straddling a domain edge do not diverge): the slot population k is read
// from (src) and written to (dst), and phi of a neighbour in a phi array (mirror ghost
// across walls).
template <int MODE>
struct AddrWrap {
    Nbr nb;
    int self;
    __device__ __forceinline__ Slot src(int k, int ex, int ey, int ez) const { return src_slot<MODE>(k, ex, ey, ez, nb, self); }
    __device__ __forceinline__ Slot dst(int k, int ex, int ey, int ez) const { return dst_slot<MODE>(k, ex, ey, ez, nb, self); }
    template <class R>
    __device__ __forceinline__ R phi(const R* __restrict__ f, int dx, int dy, int dz) const;
};

// Incoming populations of one node and their moments (steps a1-a3 of one node).
// The rest populations h_0 are stored shifted by c_0^eq (a constant shift commutes with
// the BGK relaxation of Eq. 50), so sum_k h_k gives dc = c - c_0^eq without the
// rounding of a ~0.4 composition that would swamp mu after the closure's cancellation.
template <class T, int LAT, bool FLOW>
struct Node {
    using R = typename RealOf<T>::type;
    static constexpr int Q = Scalar<LAT>::Q;
    R g[Q], hA[Q], hB[Q];
    R f[FLOW ? 19 : 1];
    R phit, dcA, dcB, S;

    template <class Addr>
    __device__ __forceinline__ void gather_scalars(const StateView& st, const Addr& ad, const DevParams& P) {
        const T* G = static_cast<const T*>(st.g);
        const T* HA = static_cast<const T*>(st.hA);
        const T* HB = static_cast<const T*>(st.hB);
        const float* rg = st.rest;
        const float* ra = st.rest ? st.rest + P.plane : nullptr;
        const float* rb = st.rest ? st.rest + 2 * P.plane : nullptr;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const Slot s = ad.src(k, Scalar<LAT>::ex(k), Scalar<LAT>::ey(k), Scalar<LAT>::ez(k));
            g[k] = load_scalar<T, SET_G, LAT>(G, rg, k, s, P);
            hA[k] = load_scalar<T, SET_H, LAT>(HA, ra, k, s, P);
            hB[k] = load_scalar<T, SET_H, LAT>(HB, rb, k, s, P);
        }
    }
    template <class Addr>
    __device__ __forceinline__ void gather_flow(const StateView& st, const Addr& ad, const DevParams& P) {
        if constexpr (FLOW) {
            const T* F = static_cast<const T*>(st.f);
#pragma unroll
            for (int k = 0; k < 19; ++k) {
                const Slot s = ad.src(k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k));
                if (is16<T>() && k == 0) f[0] = st.rest[3 * P.plane + s.node];
                else f[k] = Codec<T>::template load<SET_F>(F + (long long)s.slot * P.plane + s.node, D3Q19::w(k), P);
            }
        }
    }
    template <class Addr>
    __device__ __forceinline__ void gather(const StateView& st, const Addr& ad, const DevParams& P) {
        gather_scalars(st, ad, P);
        gather_flow(st, ad, P);
    }

    // Eq. 49 without the source, Eq. 52 (as c - c_0^eq), Eq. 33 at phi~ and Eq. 35
    __device__ __forceinline__ void moments(const DevParams& P) {
        phit = R(0); dcA = R(0); dcB = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) { phit += g[k]; dcA += hA[k]; dcB += hB[k]; }
        const R pt = interp_p(phit);
        S = source(phit, closure_dev(dcA, pt, 0, P), closure_dev(dcB, pt, 1, P), P);
    }
    __device__ __forceinline__ R phi() const { return phit + R(0.5) * S; }
    __device__ __forceinline__ R cA(const DevParams& P) const { return dcA + R(P.c0[0]); }
    __device__ __forceinline__ R cB(const DevParams& P) const { return dcB + R(P.c0[1]); }
};

// phi at x + e from a phi array: periodic wrap, mirror ghost across walls (zero normal gradient).
template <class R>
__device__ __forceinline__ R phi_at(const R* __restrict__ phi, const Nbr& nb, int dx, int dy, int dz) {
    // both candidates are indexed with constants (dx, dy, dz are unrolled), so Nbr stays in registers
    const int xx = nb.c[0][dx + 1] >= 0 ? nb.c[0][dx + 1] : nb.c[0][1];
    const int r = nb.c[2][dz + 1] >= 0 ? nb.row[dz + 1][dy + 1] : nb.row[1][dy + 1];
    return phi[r + xx];
}

template <int MODE>
template <class R>
__device__ __forceinline__ R AddrWrap<MODE>::phi(const R* __restrict__ f, int dx, int dy, int dz) const {
    return phi_at(f, nb, dx, dy, dz);
}

// Eqs. 42-45 regrouped over opposite pairs: grad = 3 sum_k w_k e_k phi(x+e_k),
// lap = 6 sum_k w_k (phi(x+e_k) - phi(x)), k = 1..18 of D3Q19. ``get(dx, dy, dz)`` returns
// phi at the neighbour (with the wall mirror already applied).
template <class R, class Get>
__device__ __forceinline__ void stencil(Get get, R phic, R& gx, R& gy, R& gz, R& lap) {
    gx = gy = gz = lap = R(0);
#pragma unroll
    for (int k = 1; k < 19; ++k) {
        const R v = get(D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k));
        const R w = R(D3Q19::w(k));
        if (D3Q19::ex(k)) gx += w * R(D3Q19::ex(k)) * v;
        if (D3Q19::ey(k)) gy += w * R(D3Q19::ey(k)) * v;
        if (D3Q19::ez(k)) gz += w * R(D3Q19::ez(k)) * v;
        lap += w * (v - phic);
    }
    gx *= R(3); gy *= R(3); gz *= R(3); lap *= R(6);
}

// Total force (Eq. 34 + Boussinesq) and velocity (Eq. 41).
template <class R>
__device__ __forceinline__ void force_velocity(const R* f, R phi, R gx, R gy, R gz, R lap, const DevParams& P,
                                               R& Fx, R& Fy, R& Fz, R& ux, R& uy, R& uz) {
    const R br = R(P.sw15) * (dwell_d(phi) * R(P.inv_W2) - lap);
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

// correctly rounded reciprocal (one MUFU-based sequence instead of a full division in FP32)
__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }

// Collisions of one node (steps a6-a8) and the scatter of the post-collision values.
template <class T, int LAT, bool FLOW, class Addr>
__device__ __forceinline__ void collide_store(const Node<T, LAT, FLOW>& nd, typename RealOf<T>::type phi,
                                              typename RealOf<T>::type ux, typename RealOf<T>::type uy,
                                              typename RealOf<T>::type uz, typename RealOf<T>::type Fx,
                                              typename RealOf<T>::type Fy, typename RealOf<T>::type Fz,
                                              const StateView& out, const Addr& ad, const DevParams& P) {
    const int self = ad.self;
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    constexpr int Q = L::Q;
    if constexpr (FLOW) {
        // Eqs. 36-39: He-Shan-Doolen forcing, He-Luo equilibrium shifted by -F_k/2
        R ph = R(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) ph += nd.f[k];
        const R usq = ux * ux + uy * uy + uz * uz;
        const R omf = R(P.om_f);
        T* F = static_cast<T*>(out.f);
        R f0post = R(0), resid = R(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const R w = R(D3Q19::w(k));
            const R cu = R(D3Q19::ex(k)) * ux + R(D3Q19::ey(k)) * uy + R(D3Q19::ez(k)) * uz;
            const R gam = w * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
            const R Fk = gam * ((R(D3Q19::ex(k)) - ux) * Fx + (R(D3Q19::ey(k)) - uy) * Fy + (R(D3Q19::ez(k)) - uz) * Fz);
            const R feq = w * (ph + cu + R(1.5) * cu * cu - R(0.5) * usq) - R(0.5) * Fk;
            const R post = nd.f[k] - omf * (nd.f[k] - feq) + Fk;
            const Slot s = ad.dst(k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k));
            if (is16<T>() && k == 0) { f0post = post; continue; }
            resid += Codec<T>::template store_residual<SET_F>(F + (long long)s.slot * P.plane + s.node, post,
                                                              D3Q19::w(k), P);
        }
        if (is16<T>()) out.rest[3 * P.plane + self] = float(f0post + resid);
    }
    const R S = nd.S;
    const R p = interp_p(phi);
    const R muA = closure_dev(nd.dcA, p, 0, P);
    const R muB = closure_dev(nd.dcB, p, 1, P);
    const R inv_cs2 = R(L::cs2() == 0.25 ? 4.0 : 3.0);
    const R omg = R(P.om_g);
    // Eqs. 50-51 with M^alpha(phi) of §2.3 and tau_h = M / c_s^2
    const R MA = R(P.M0[0]) * (R(1) - phi) + R(P.M1[0]) * phi;
    const R MB = R(P.M0[1]) * (R(1) - phi) + R(P.M1[1]) * phi;
    const R omA = recip(MA * inv_cs2 + R(0.5));
    const R omB = recip(MB * inv_cs2 + R(0.5));
    T* G = static_cast<T*>(out.g);
    T* HA = static_cast<T*>(out.hA);
    T* HB = static_cast<T*>(out.hB);
    float* rg = out.rest;
    float* ra = out.rest ? out.rest + P.plane : nullptr;
    float* rb = out.rest ? out.rest + 2 * P.plane : nullptr;
    R g0 = R(0), hA0 = R(0), hB0 = R(0);          // rest populations, stored last
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const R w = R(L::w(k));
        const R cu = R(L::ex(k)) * ux + R(L::ey(k)) * uy + R(L::ez(k)) * uz;
        // Eqs. 46-48
        const R geq = w * phi * (R(1) + inv_cs2 * cu) - R(0.5) * w * S;
        const R gpost = nd.g[k] - omg * (nd.g[k] - geq) + w * S;
        R heqA, heqB;
        if (k == 0) {                      // shifted by c_0^eq like the stored h_0
            heqA = nd.dcA - (R(1) - w) * muA;
            heqB = nd.dcB - (R(1) - w) * muB;
        } else {
            heqA = w * muA + w * nd.cA(P) * inv_cs2 * cu;
            heqB = w * muB + w * nd.cB(P) * inv_cs2 * cu;
        }
        const R hApost = nd.hA[k] - omA * (nd.hA[k] - heqA);
        const R hBpost = nd.hB[k] - omB * (nd.hB[k] - heqB);
        if (k == 0) { g0 = gpost; hA0 = hApost; hB0 = hBpost; continue; }
        const Slot s = ad.dst(k, L::ex(k), L::ey(k), L::ez(k));
        // 16-bit storage: rounding residuals of the moving populations go to the rest population
        g0 += store_moving<T, SET_G, LAT>(G, k, s, gpost, P);
        hA0 += store_moving<T, SET_H, LAT>(HA, k, s, hApost, P);
        hB0 += store_moving<T, SET_H, LAT>(HB, k, s, hBpost, P);
    }
    const Slot s0{self, 0};
    store_scalar<T, SET_G, LAT>(G, rg, 0, s0, g0, P);
    store_scalar<T, SET_H, LAT>(HA, ra, 0, s0, hA0, P);
    store_scalar<T, SET_H, LAT>(HB, rb, 0, s0, hB0, P);
}

// ------------------------------------------------------------------------------------
// One coupled step per node. With flow the phi field of this step must already be in
// phi_field (phi pass); MODE AA_* works in place on ``st``, PULL reads ``st`` and writes ``out``.
template <class T, int LAT, bool FLOW, int MODE>
__global__ void __launch_bounds__(kBlockX)
step_kernel(const DevParams P, const StateView st, const StateView out,
            const typename RealOf<T>::type* __restrict__ phi_field) {
    using R = typename RealOf<T>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int self = node_of(x, y, z, P);
    AddrWrap<MODE> ad;
    ad.self = self;
    ad.nb.init(x, y, z, P);
    Node<T, LAT, FLOW> nd;
    nd.gather(st, ad, P);
    nd.moments(P);
    R phi;
    if constexpr (FLOW) phi = phi_field[self]; else phi = nd.phi();
    R ux = R(0), uy = R(0), uz = R(0), Fx = R(0), Fy = R(0), Fz = R(0);
    if constexpr (FLOW) {
        R gx, gy, gz, lap;
        stencil([&](int dx, int dy, int dz) { return ad.phi(phi_field, dx, dy, dz); }, phi, gx, gy, gz, lap);
        force_velocity(nd.f, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
    }
    collide_store(nd, phi, ux, uy, uz, Fx, Fy, Fz, out, ad, P);
}

// phi = sum g + S/2 of every node (Eq. 49), read by the capillary stencil.
template <class T, int LAT, int MODE>
__global__ void __launch_bounds__(kBlockX)
phi_kernel(const DevParams P, const StateView st, typename RealOf<T>::type* __restrict__ phi_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int self = node_of(x, y, z, P);
    AddrWrap<MODE> ad;
    ad.self = self;
    ad.nb.init(x, y, z, P);
    Node<T, LAT, false> nd;
    nd.gather_scalars(st, ad, P);
    nd.moments(P);
    phi_out[self] = nd.phi();
}

// ------------------------------------------------------------------------------------
// Fused two-buffer flow step: each CTA marches an (FX x FY) column of (x, y) through a
// chunk of z planes. At each plane z:
//   fill(z + 1): every thread gathers the scalar populations (g, h^A, h^B) of its own
//     column at plane z + 1, keeps them decoded in shared memory (double-buffered) with
//     S and c - c_0^eq, and writes phi into a 3-plane ring; 84 threads add the ring's
//     one-node halo.
//   centre(z): gather the 19 f populations, take the scalar populations of plane z from
//     shared memory, form the capillary stencil from the ring, collide and store f, then
//     collide and store g, h^A, h^B (all stores local and coalesced).
// The stencil therefore needs no separate pass and the scalar populations are read from
// HBM once; the halo re-reads hit L2.
constexpr int FX = 32, FY = 8, FT = FX * FY;
constexpr int kHalo = 2 * (FX + 2) + 2 * FY;    // ring positions outside the tile (84)
constexpr int kSPops = 3 * 7 + 3;               // 21 scalar populations + S, dcA, dcB

template <class R>
__host__ __device__ constexpr size_t fused_smem_bytes() {
    return sizeof(R) * (3 * (FY + 2) * (FX + 2) + 2 * kSPops * FT);
}

template <class T>
__global__ void __launch_bounds__(FT, sizeof(typename RealOf<T>::type) == 8 ? 1 : 3)
fused_flow_kernel(const DevParams P, const StateView src, const StateView dst, int zchunk) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT_D3Q7>;
    constexpr int Q = L::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R (*ring)[FY + 2][FX + 2] = reinterpret_cast<R (*)[FY + 2][FX + 2]>(smem_raw);
    R* spops = reinterpret_cast<R*>(smem_raw) + 3 * (FY + 2) * (FX + 2);   // [2][kSPops][FT]
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * FX + tx;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * FY;
    const int zs = blockIdx.z * zchunk;
    const int ze = min(zs + zchunk, P.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < P.nx && y < P.ny;

    // domain position of ring position (hx, hy): periodic wrap in x and y, mirror across x walls
    auto wrap_xy = [&](int hx, int hy, int& gx, int& gy) {
        gx = x0 + hx;
        gy = y0 + hy;
        if (gx < 0) gx = P.wall_x ? 0 : gx + P.nx;
        else if (gx >= P.nx) gx = P.wall_x ? P.nx - 1 : gx - P.nx;
        if (gy < 0) gy += P.ny;
        else if (gy >= P.ny) gy -= P.ny;
        return gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny;
    };
    auto zwrap = [&](int zz) {
        if (zz < 0) return P.wall_z ? 0 : zz + P.nz;
        if (zz >= P.nz) return P.wall_z ? P.nz - 1 : zz - P.nz;
        return zz;
    };
    // phi (and, for a tile node, its scalar populations in buffer buf) of plane zz
    auto fill = [&](int zz, int s, int buf) {
        const int zr = zwrap(zz);
        {
            int gx, gy;
            R v = R(0);
            if (wrap_xy(tx, ty, gx, gy)) {
                AddrWrap<PULL> ad;
                ad.self = node_of(gx, gy, zr, P);
                ad.nb.init(gx, gy, zr, P);
                Node<T, LAT_D3Q7, false> nd;
                nd.gather_scalars(src, ad, P);
                nd.moments(P);
                v = nd.phi();
                if (active && buf >= 0) {
                    R* sp = spops + buf * kSPops * FT + tid;
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        sp[k * FT] = nd.g[k];
                        sp[(Q + k) * FT] = nd.hA[k];
                        sp[(2 * Q + k) * FT] = nd.hB[k];
                    }
                    sp[(3 * Q) * FT] = nd.S;
                    sp[(3 * Q + 1) * FT] = nd.dcA;
                    sp[(3 * Q + 2) * FT] = nd.dcB;
                }
            }
            ring[s][ty + 1][tx + 1] = v;
        }
        if (tid < kHalo) {
            int hx, hy;
            if (tid < FX + 2) { hx = tid - 1; hy = -1; }
            else if (tid < 2 * (FX + 2)) { hx = tid - (FX + 2) - 1; hy = FY; }
            else if (tid < 2 * (FX + 2) + FY) { hx = -1; hy = tid - 2 * (FX + 2); }
            else { hx = FX; hy = tid - 2 * (FX + 2) - FY; }
            int gx, gy;
            R v = R(0);
            if (wrap_xy(hx, hy, gx, gy)) {
                AddrWrap<PULL> ad;
                ad.self = node_of(gx, gy, zr, P);
                ad.nb.init(gx, gy, zr, P);
                Node<T, LAT_D3Q7, false> nd;
                nd.gather_scalars(src, ad, P);
                nd.moments(P);
                v = nd.phi();
            }
            ring[s][hy + 1][hx + 1] = v;
        }
    };

    int sp = 0, sc = 1, sn = 2;   // ring slots of planes z - 1, z, z + 1
    fill(zs - 1, sp, -1);
    fill(zs, sc, zs & 1);
    for (int z = zs; z < ze; ++z) {
        fill(z + 1, sn, (z + 1) & 1);
        __syncthreads();
        if (active) {
            AddrWrap<PULL> ad;
            ad.self = node_of(x, y, z, P);
            ad.nb.init(x, y, z, P);
            Node<T, LAT_D3Q7, true> nd;
            nd.gather_flow(src, ad, P);
            const R* spc = spops + (z & 1) * kSPops * FT + tid;
            nd.S = spc[(3 * Q) * FT];
            nd.dcA = spc[(3 * Q + 1) * FT];
            nd.dcB = spc[(3 * Q + 2) * FT];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                nd.g[k] = spc[k * FT];
                nd.hA[k] = spc[(Q + k) * FT];
                nd.hB[k] = spc[(2 * Q + k) * FT];
            }
            const R phi = ring[sc][ty + 1][tx + 1];
            R gx, gy, gz, lap, Fx, Fy, Fz, ux, uy, uz;
            stencil([&](int dx, int dy, int dz) {
                        const int s = dz < 0 ? sp : (dz > 0 ? sn : sc);
                        return ring[s][ty + 1 + dy][tx + 1 + dx];
                    }, phi, gx, gy, gz, lap);
            force_velocity(nd.f, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
            collide_store(nd, phi, ux, uy, uz, Fx, Fy, Fz, dst, ad, P);
        }
        __syncthreads();
        const int t = sp; sp = sc; sc = sn; sn = t;
    }
}

// ------------------------------------------------------------------------------------
// Initial populations at rest, computed in FP64 then stored. MODE AA_EVEN writes the
// incoming populations in their own slots (time 0 of the AA pattern); MODE PULL writes
// what a pull gather must find: slot k of node y holds the initial population k of node
// y + e_k, or, beyond a wall, the initial population opp(k) of y itself.
enum { INIT_G = 0, INIT_HA = 1, INIT_HB = 2, INIT_F = 3 };

template <int LAT>
__device__ __forceinline__ double init_value(int set, int k, int node, const Nbr& nb,
                                             const double* __restrict__ phi0, const double* __restrict__ cA0,
                                             const double* __restrict__ cB0, const DevParams& P) {
    const double ph = phi0[node];
    if (set == INIT_F) {
        double gx, gy, gz, lap;
        stencil([&](int dx, int dy, int dz) { return phi_at(phi0, nb, dx, dy, dz); }, ph, gx, gy, gz, lap);
        const double br = P.sw15 * (dwell_d(ph) * P.inv_W2 - lap);
        const double Fx = br * gx + ph * P.g[0], Fy = br * gy + ph * P.g[1], Fz = br * gz + ph * P.g[2];
        const double w = D3Q19::w(k);
        return -0.5 * w * (D3Q19::ex(k) * Fx + D3Q19::ey(k) * Fy + D3Q19::ez(k) * Fz);   // Eqs. 37-39
    }
    const double pp = interp_p(ph);
    const double dA = cA0[node] - P.c0[0], dB = cB0[node] - P.c0[1];
    const double muA = closure_dev(dA, pp, 0, P), muB = closure_dev(dB, pp, 1, P);
    const double w = Scalar<LAT>::w(k);
    if (set == INIT_G) return w * ph - 0.5 * w * source(ph, muA, muB, P);             // Eq. 47, u = 0
    const double d = set == INIT_HA ? dA : dB, mu = set == INIT_HA ? muA : muB;       // Eq. 51, u = 0
    return k == 0 ? d - (1.0 - w) * mu : w * mu;                                      // h_0 shifted by c_0^eq
}

template <class T, int LAT, bool FLOW, int MODE>
__global__ void __launch_bounds__(kBlockX)
init_kernel(const DevParams P, const StateView st, const double* __restrict__ phi0,
            const double* __restrict__ cA0, const double* __restrict__ cB0) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int self = node_of(x, y, z, P);
    Nbr nb;
    nb.init(x, y, z, P);
    T* G = static_cast<T*>(st.g);
    T* HA = static_cast<T*>(st.hA);
    T* HB = static_cast<T*>(st.hB);
    float* rg = st.rest;
    float* ra = st.rest ? st.rest + P.plane : nullptr;
    float* rb = st.rest ? st.rest + 2 * P.plane : nullptr;
    // which node's initial population (and which index) slot k of this node holds
    auto source_of = [&](int k, int ex, int ey, int ez, int& node, int& kk, Nbr& snb) {
        node = self; kk = k; snb = nb;
        if (MODE == PULL && k != 0) {
            int q;
            if (nb.at(ex, ey, ez, self, q)) {
                node = q;
                snb.init(nb.c[0][ex + 1], nb.c[1][ey + 1], nb.c[2][ez + 1], P);
            } else {
                kk = opp(k);
            }
        }
    };
#pragma unroll 1
    for (int k = 0; k < L::Q; ++k) {
        int node; int kk; Nbr snb;
        source_of(k, L::ex(k), L::ey(k), L::ez(k), node, kk, snb);
        const Slot s{self, k};
        store_scalar<T, SET_G, LAT>(G, rg, k, s, R(init_value<LAT>(INIT_G, kk, node, snb, phi0, cA0, cB0, P)), P);
        store_scalar<T, SET_H, LAT>(HA, ra, k, s, R(init_value<LAT>(INIT_HA, kk, node, snb, phi0, cA0, cB0, P)), P);
        store_scalar<T, SET_H, LAT>(HB, rb, k, s, R(init_value<LAT>(INIT_HB, kk, node, snb, phi0, cA0, cB0, P)), P);
    }
    if constexpr (FLOW) {
        T* F = static_cast<T*>(st.f);
#pragma unroll 1
        for (int k = 0; k < 19; ++k) {
            int node; int kk; Nbr snb;
            source_of(k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k), node, kk, snb);
            const R v = R(init_value<LAT>(INIT_F, kk, node, snb, phi0, cA0, cB0, P));
            if (is16<T>() && k == 0) st.rest[3 * P.plane + self] = float(v);
            else Codec<T>::template store<SET_F>(F + (long long)k * P.plane + self, v, D3Q19::w(k), P);
        }
    }
}

// Macroscopic fields of the current time level (phi_field filled by the phi pass with flow).
template <class T, int LAT, bool FLOW, int MODE>
__global__ void __launch_bounds__(kBlockX)
fields_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ phi_field,
              FieldPtrs out) {
    using R = typename RealOf<T>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int self = node_of(x, y, z, P);
    AddrWrap<MODE> ad;
    ad.nb.init(x, y, z, P);
    ad.self = self;
    Node<T, LAT, FLOW> nd;
    nd.gather(st, ad, P);
    nd.moments(P);
    R phi;
    if constexpr (FLOW) phi = phi_field[self]; else phi = nd.phi();
    const R p = interp_p(phi);
    R vals[LBM_NFIELDS_DEV];
    vals[0] = phi;
    vals[1] = closure_dev(nd.dcA, p, 0, P);
    vals[2] = closure_dev(nd.dcB, p, 1, P);
    vals[3] = nd.cA(P);
    vals[4] = nd.cB(P);
    vals[5] = R(0); vals[6] = R(0); vals[7] = R(0); vals[8] = R(0);
    vals[9] = nd.S;
    if constexpr (FLOW) {
        R gx, gy, gz, lap, Fx, Fy, Fz;
        stencil([&](int dx, int dy, int dz) { return ad.phi(phi_field, dx, dy, dz); }, phi, gx, gy, gz, lap);
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
template <class T, int LAT, bool FLOW, int MODE>
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
        AddrWrap<MODE> ad;
        ad.nb.init(x, y, z, P);
        ad.self = int(id);
        Node<T, LAT, FLOW> nd;
        nd.gather(st, ad, P);
        nd.moments(P);
        R phi;
        if constexpr (FLOW) phi = phi_field[id]; else phi = nd.phi();
        double umag = 0.0, ph = 0.0;
        if constexpr (FLOW) {
            R gx, gy, gz, lap, Fx, Fy, Fz, ux, uy, uz;
            stencil([&](int dx, int dy, int dz) { return ad.phi(phi_field, dx, dy, dz); }, phi, gx, gy, gz, lap);
            force_velocity(nd.f, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
            umag = sqrt(double(ux) * ux + double(uy) * uy + double(uz) * uz);
            R s = R(0);
#pragma unroll
            for (int k = 0; k < 19; ++k) s += nd.f[k];
            ph = s;
        }
        const double vals[5] = {double(phi), double(nd.dcA) + P.c0[0], double(nd.dcB) + P.c0[1], ph,
                                double(nd.S)};
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
            const double u = __shfl_down_sync(0xffffffffu, v, o);
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
                const double u = __shfl_down_sync(0xffffffffu, v, o);
                v = (i == 5) ? fmax(v, u) : v + u;
            }
            if (lane == 0) partials[(long long)blockIdx.x * LBM_NRED_DEV + i] = v;
        }
    }
}

// ------------------------------------------------------------------------------------
// Host launchers for one storage type. ``mode`` is AA_EVEN / AA_ODD for the in-place
// layout and PULL for the two-buffer layout (st = the current state buffer).
inline dim3 node_grid(const DevParams& P, int& bx) {
    bx = P.nx >= kBlockX ? kBlockX : ((P.nx + 31) / 32) * 32;
    return dim3((P.nx + bx - 1) / bx, P.ny, P.nz);
}

#define LBM_MODE_SWITCH(MODE_VAR, ...)                                          \
    switch (MODE_VAR) {                                                         \
        case AA_EVEN: { constexpr int M = AA_EVEN; __VA_ARGS__; } break;        \
        case AA_ODD: { constexpr int M = AA_ODD; __VA_ARGS__; } break;          \
        default: { constexpr int M = PULL; __VA_ARGS__; } break;                \
    }

template <class T>
struct Launchers {
    using R = typename RealOf<T>::type;

    template <int LAT, bool FLOW>
    static void init(const DevParams& P, const StateView& st, bool pull, const double* phi0, const double* cA0,
                     const double* cB0, cudaStream_t s) {
        int bx; const dim3 grid = node_grid(P, bx);
        if (pull) init_kernel<T, LAT, FLOW, PULL><<<grid, bx, 0, s>>>(P, st, phi0, cA0, cB0);
        else init_kernel<T, LAT, FLOW, AA_EVEN><<<grid, bx, 0, s>>>(P, st, phi0, cA0, cB0);
    }
    template <int LAT>
    static void phi(const DevParams& P, const StateView& st, int mode, void* phi_work, cudaStream_t s) {
        int bx; const dim3 grid = node_grid(P, bx);
        R* ph = static_cast<R*>(phi_work);
        LBM_MODE_SWITCH(mode, phi_kernel<T, LAT, M><<<grid, bx, 0, s>>>(P, st, ph));
    }
    // the per-node step kernel; with flow, the phi pass of the same step must precede it
    template <int LAT, bool FLOW>
    static void step(const DevParams& P, const StateView& st, const StateView& out, int mode, void* phi_work,
                     cudaStream_t s) {
        int bx; const dim3 grid = node_grid(P, bx);
        R* phi = static_cast<R*>(phi_work);
        LBM_MODE_SWITCH(mode, step_kernel<T, LAT, FLOW, M><<<grid, bx, 0, s>>>(P, st, out, phi));
    }
    static void fused(const DevParams& P, const StateView& src, const StateView& dst, int zchunk, cudaStream_t s) {
        const dim3 block(FX, FY);
        const dim3 grid((P.nx + FX - 1) / FX, (P.ny + FY - 1) / FY, (P.nz + zchunk - 1) / zchunk);
        constexpr size_t smem = fused_smem_bytes<R>();
        // opt in to more than 48 KB of dynamic shared memory, once per device (a repeated
        // call from a racing thread is harmless)
        static unsigned long long configured = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !(configured & (1ull << dev))) {
            cudaFuncSetAttribute(fused_flow_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            configured |= 1ull << dev;
        }
        fused_flow_kernel<T><<<grid, block, smem, s>>>(P, src, dst, zchunk);
    }
    template <int LAT, bool FLOW>
    static void fields(const DevParams& P, const StateView& st, int mode, void* phi_work, FieldPtrs out,
                       cudaStream_t s) {
        int bx; const dim3 grid = node_grid(P, bx);
        R* phi = static_cast<R*>(phi_work);
        if constexpr (FLOW) { LBM_MODE_SWITCH(mode, phi_kernel<T, LAT, M><<<grid, bx, 0, s>>>(P, st, phi)); }
        LBM_MODE_SWITCH(mode, fields_kernel<T, LAT, FLOW, M><<<grid, bx, 0, s>>>(P, st, phi, out));
    }
    template <int LAT, bool FLOW>
    static void reduce(const DevParams& P, const StateView& st, int mode, void* phi_work, double* partials,
                       int nblocks, cudaStream_t s) {
        R* phi = static_cast<R*>(phi_work);
        if constexpr (FLOW) {
            int bx; const dim3 grid = node_grid(P, bx);
            LBM_MODE_SWITCH(mode, phi_kernel<T, LAT, M><<<grid, bx, 0, s>>>(P, st, phi));
        }
        LBM_MODE_SWITCH(mode, reduce_kernel<T, LAT, FLOW, M><<<nblocks, 256, 0, s>>>(P, st, phi, partials));
    }
};

// Dispatch over (lattice, flow) for one storage type.
#define LBM_DEFINE_LAUNCHERS(T, SUFFIX)                                                                   \
    void launch_init_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, bool pull,      \
                              const double* a, const double* b, const double* c, cudaStream_t s) {        \
        if (lat == LAT_D2Q5) Launchers<T>::init<LAT_D2Q5, false>(P, st, pull, a, b, c, s);                 \
        else if (flow) Launchers<T>::init<LAT_D3Q7, true>(P, st, pull, a, b, c, s);                        \
        else Launchers<T>::init<LAT_D3Q7, false>(P, st, pull, a, b, c, s);                                 \
    }                                                                                                     \
    void launch_phi_##SUFFIX(const DevParams& P, const StateView& st, int lat, int mode, void* phi,       \
                             cudaStream_t s) {                                                            \
        if (lat == LAT_D2Q5) Launchers<T>::phi<LAT_D2Q5>(P, st, mode, phi, s);                             \
        else Launchers<T>::phi<LAT_D3Q7>(P, st, mode, phi, s);                                             \
    }                                                                                                     \
    void launch_step_##SUFFIX(const DevParams& P, const StateView& st, const StateView& out, int lat,     \
                              bool flow, int mode, void* phi, cudaStream_t s) {                            \
        if (lat == LAT_D2Q5) Launchers<T>::step<LAT_D2Q5, false>(P, st, out, mode, phi, s);                \
        else if (flow) Launchers<T>::step<LAT_D3Q7, true>(P, st, out, mode, phi, s);                       \
        else Launchers<T>::step<LAT_D3Q7, false>(P, st, out, mode, phi, s);                                \
    }                                                                                                     \
    void launch_fused_##SUFFIX(const DevParams& P, const StateView& src, const StateView& dst, int zchunk, \
                               cudaStream_t s) {                                                          \
        Launchers<T>::fused(P, src, dst, zchunk, s);                                                      \
    }                                                                                                     \
    void launch_fields_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, int mode,    \
                                void* phi, FieldPtrs out, cudaStream_t s) {                               \
        if (lat == LAT_D2Q5) Launchers<T>::fields<LAT_D2Q5, false>(P, st, mode, phi, out, s);              \
        else if (flow) Launchers<T>::fields<LAT_D3Q7, true>(P, st, mode, phi, out, s);                     \
        else Launchers<T>::fields<LAT_D3Q7, false>(P, st, mode, phi, out, s);                              \
    }                                                                                                     \
    void launch_reduce_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, int mode,    \
                                void* phi, double* partials, int nblocks, cudaStream_t s) {               \
        if (lat == LAT_D2Q5) Launchers<T>::reduce<LAT_D2Q5, false>(P, st, mode, phi, partials, nblocks, s); \
        else if (flow) Launchers<T>::reduce<LAT_D3Q7, true>(P, st, mode, phi, partials, nblocks, s);       \
        else Launchers<T>::reduce<LAT_D3Q7, false>(P, st, mode, phi, partials, nblocks, s);                \
    }

}  // namespace lbm
