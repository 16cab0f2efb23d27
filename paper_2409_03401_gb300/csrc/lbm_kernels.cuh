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

#include <type_traits>

namespace lbm {

constexpr int kBlockX = 128;
enum { AA_EVEN = 0, AA_ODD = 1, PULL = 2 };

// Wrapped neighbour coordinates of one node. c[a][1 + d] is the coordinate x_a + d along
// axis a (d = -1, 0, 1) after the periodic wrap, or -1 where x_a + d lies beyond a wall;
// row[iz][iy] = (z' ny + y') nx of the neighbouring rows (own plane beyond a wall). All
// selects, no branches: warps straddling a domain edge do not diverge. init_xy() once per
// (x, y) column and set_z() per plane let z-marching kernels skip the x/y part.
struct Nbr {
    int c[3][3];
    int row[3][3];
    __device__ __forceinline__ static int wrap(int q, int n, int wall) {
        return q < 0 ? (wall ? -1 : q + n) : (q >= n ? (wall ? -1 : q - n) : q);
    }
    __device__ __forceinline__ void init_xy(int x, int y, const DevParams& P) {
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            c[0][d + 1] = wrap(x + d, P.nx, P.wall_x);
            c[1][d + 1] = wrap(y + d, P.ny, 0);
        }
    }
    __device__ __forceinline__ static int wrap2(int q, int n, int wall_lo, int wall_hi) {
        return q < 0 ? (wall_lo ? -1 : q + n) : (q >= n ? (wall_hi ? -1 : q - n) : q);
    }
    __device__ __forceinline__ void set_z(int z, const DevParams& P) {
#pragma unroll
        for (int d = -1; d <= 1; ++d) c[2][d + 1] = wrap2(z + d, P.nz, P.wall_zlo, P.wall_zhi);
#pragma unroll
        for (int iz = 0; iz < 3; ++iz)
#pragma unroll
            for (int iy = 0; iy < 3; ++iy)
                row[iz][iy] = ((c[2][iz] < 0 ? z : c[2][iz]) * P.ny + c[1][iy]) * P.nx;
    }
    __device__ __forceinline__ void init(int x, int y, int z, const DevParams& P) {
        init_xy(x, y, P);
        set_z(z, P);
    }
    // node x + (dx, dy, dz); false (and the node itself) when that lies beyond a wall
    __device__ __forceinline__ bool at(int dx, int dy, int dz, int self, int& out) const {
        const int xx = c[0][dx + 1], zz = c[2][dz + 1];
        const bool in = (dx == 0 || xx >= 0) && (dz == 0 || zz >= 0);
        out = in ? row[dz + 1][dy + 1] + xx : self;
        return in;
    }
};

// Slot population k of node self is read from / written to in each streaming mode. Across a
// wall both fall back to the node itself with k and opp(k) exchanged (half-way bounce-back).
template <int MODE>
struct Addr {
    // FP32 rest plane of f read (written) by a step in this mode with 16-bit storage: the
    // two-buffer layout keeps f_0 in plane 3 of each copy; in place, time levels alternate
    // between planes 3 (even) and 4 (odd), because neighbours read a node's f_0 as the
    // reference of the populations it wrote (Codec16Pop) while the node replaces it.
    static constexpr int kF0In = MODE == AA_ODD ? 4 : 3;
    static constexpr int kF0Out = MODE == AA_EVEN ? 4 : 3;
    Nbr nb;
    int self;
    __device__ __forceinline__ Slot src(int k, int ex, int ey, int ez) const {
        if (MODE == AA_EVEN || k == 0) return {self, k};
        int q;
        const bool in = nb.at(-ex, -ey, -ez, self, q);
        if (MODE == AA_ODD) return in ? Slot{q, opp(k)} : Slot{self, k};
        return in ? Slot{q, k} : Slot{self, opp(k)};
    }
    __device__ __forceinline__ Slot dst(int k, int ex, int ey, int ez) const {
        if (k == 0 || MODE == PULL) return {self, k};
        if (MODE == AA_EVEN) return {self, opp(k)};
        int q;
        return nb.at(ex, ey, ez, self, q) ? Slot{q, k} : Slot{self, opp(k)};
    }
    // node that stored the population gathered as k: x - e_k (its outgoing k), or the node
    // itself across a wall (its outgoing opp(k), bounced back)
    __device__ __forceinline__ int writer(int k, int ex, int ey, int ez) const {
        if (k == 0) return self;
        if (MODE == AA_EVEN) {
            int q;
            nb.at(-ex, -ey, -ez, self, q);
            return q;
        }
        return src(k, ex, ey, ez).node;
    }
    // phi of a neighbour in a phi array, mirror ghost across walls (zero normal gradient)
    template <class R>
    __device__ __forceinline__ R phi(const R* __restrict__ f, int dx, int dy, int dz) const {
        const int xx = nb.c[0][dx + 1] >= 0 ? nb.c[0][dx + 1] : nb.c[0][1];
        const int r = nb.c[2][dz + 1] >= 0 ? nb.row[dz + 1][dy + 1] : nb.row[1][dy + 1];
        return f[r + xx];
    }
};

// Pull addressing at a node whose whole neighbourhood (one node in x and y, and in z) lies
// inside the lattice: no wrap and no wall, so the source of population k is node
// self - e_k, an offset that is the same for every thread of a block.
struct AddrInterior {
    static constexpr int kF0In = 3, kF0Out = 3;
    int self;
    int sx, sxy;   // nx, nx * ny
    __device__ __forceinline__ Slot src(int k, int ex, int ey, int ez) const {
        return {self - ex - ey * sx - ez * sxy, k};
    }
    __device__ __forceinline__ int writer(int k, int ex, int ey, int ez) const { return src(k, ex, ey, ez).node; }
    __device__ __forceinline__ Slot dst(int k, int, int, int) const { return {self, k}; }
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

    template <class A>
    __device__ __forceinline__ void gather_scalars(const StateView& st, const A& ad, const DevParams& P) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const Slot s = ad.src(k, Scalar<LAT>::ex(k), Scalar<LAT>::ey(k), Scalar<LAT>::ez(k));
            g[k] = load_scalar<T, SET_G, LAT, Planes<LAT>::G, 0>(st, k, s, P);
            hA[k] = load_scalar<T, SET_H, LAT, Planes<LAT>::HA, 1>(st, k, s, P);
            hB[k] = load_scalar<T, SET_H, LAT, Planes<LAT>::HB, 2>(st, k, s, P);
        }
    }
    // With 16-bit storage ``ref(k, ex, ey, ez, slot)`` gives f_0 / w_0 of the node that stored
    // the population gathered as k (for k = 0 of the node itself), and f_k / w_k is the stored
    // deviation, in its storage unit, plus that reference (Codec16Pop).
    template <class A, class Ref>
    __device__ __forceinline__ void gather_flow(const StateView& st, const A& ad, const DevParams& P, Ref ref) {
        if constexpr (FLOW) {
#pragma unroll
            for (int k = 0; k < 19; ++k) {
                const int ex = D3Q19::ex(k), ey = D3Q19::ey(k), ez = D3Q19::ez(k);
                const Slot s = ad.src(k, ex, ey, ez);
                if constexpr (is16<T>()) {
                    if (k == 0) f[0] = R(D3Q19::w(0)) * ref(0, 0, 0, 0, s);
                    else f[k] = fmaf(Codec<T>::template load<SET_F>(element<T, 0>(st, k, s), D3Q19::w(k), P),
                                     1.0f / Codec<T>::template unit<SET_F>(), ref(k, ex, ey, ez, s));
                } else {
                    f[k] = Codec<T>::template load<SET_F>(element<T, 0>(st, k, s), D3Q19::w(k), P);
                }
            }
        }
    }
    template <class A>
    __device__ __forceinline__ void gather_flow(const StateView& st, const A& ad, const DevParams& P) {
        const float* f0 = is16<T>() ? st.rest + A::kF0In * P.plane : nullptr;
        gather_flow(st, ad, P, [&](int k, int ex, int ey, int ez, Slot) {
            return f0[ad.writer(k, ex, ey, ez)] * float(1.0 / D3Q19::w(0));
        });
    }
    template <class A>
    __device__ __forceinline__ void gather(const StateView& st, const A& ad, const DevParams& P) {
        gather_scalars(st, ad, P);
        gather_flow(st, ad, P);
    }

    // Eq. 49 without the source, Eq. 52 (as c - c_0^eq), Eq. 33 at phi~ and Eq. 35. With
    // 16-bit storage the moving populations are values per unit weight x_k (Codec16Pop): the
    // sums weight them back, sum_k P_k = P_0 + sum_k>0 (w_k x_k + offset_k).
    __device__ __forceinline__ void moments(const DevParams& P) {
        if constexpr (is16<T>()) {
            using C = Codec<T>;
            phit = g[0] + R(0.5 * (1.0 - Scalar<LAT>::w(0)));      // sum of the offsets w_k / 2
            dcA = hA[0];
            dcB = hB[0];
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                phit += R(C::template scale<SET_G>(Scalar<LAT>::w(k))) * g[k];
                dcA += R(C::template scale<SET_H>(Scalar<LAT>::w(k))) * hA[k];
                dcB += R(C::template scale<SET_H>(Scalar<LAT>::w(k))) * hB[k];
            }
        } else {
            phit = R(0); dcA = R(0); dcB = R(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) { phit += g[k]; dcA += hA[k]; dcB += hB[k]; }
        }
        const R pt = interp_p(phit);
        S = source(phit, closure_dev(dcA, pt, 0, P), closure_dev(dcB, pt, 1, P), P);
    }
    // c - c_0^eq of both components (Eq. 52 with the shifted h_0), as in moments()
    __device__ __forceinline__ void dc_sums() {
        if constexpr (is16<T>()) {
            using C = Codec<T>;
            dcA = hA[0];
            dcB = hB[0];
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                dcA += R(C::template scale<SET_H>(Scalar<LAT>::w(k))) * hA[k];
                dcB += R(C::template scale<SET_H>(Scalar<LAT>::w(k))) * hB[k];
            }
        } else {
            dcA = R(0); dcB = R(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) { dcA += hA[k]; dcB += hB[k]; }
        }
    }
    // p_h = sum f (Eq. 40)
    __device__ __forceinline__ R flow_p() const {
        static_assert(FLOW, "flow moments of a node without flow populations");
        if constexpr (is16<T>()) {
            R ph = f[0];                                    // f_k / w_k for k > 0
#pragma unroll
            for (int k = 1; k < 19; ++k) ph += R(D3Q19::w(k)) * f[k];
            return ph;
        } else {
            R ph = R(0);
#pragma unroll
            for (int k = 0; k < 19; ++k) ph += f[k];
            return ph;
        }
    }
    // j = sum f e (Eq. 41 before the force shift)
    __device__ __forceinline__ void flow_j(R& jx, R& jy, R& jz) const {
        static_assert(FLOW, "flow moments of a node without flow populations");
        jx = jy = jz = R(0);
#pragma unroll
        for (int k = 1; k < 19; ++k) {
            R v = f[k];
            if constexpr (is16<T>()) v *= R(D3Q19::w(k));   // f_k / w_k
            if (D3Q19::ex(k)) jx += R(D3Q19::ex(k)) * v;
            if (D3Q19::ey(k)) jy += R(D3Q19::ey(k)) * v;
            if (D3Q19::ez(k)) jz += R(D3Q19::ez(k)) * v;
        }
    }
    __device__ __forceinline__ R phi() const { return phit + R(0.5) * S; }
    __device__ __forceinline__ R cA(const DevParams& P) const { return dcA + coef<R>(P).c0[0]; }
    __device__ __forceinline__ R cB(const DevParams& P) const { return dcB + coef<R>(P).c0[1]; }
};

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
template <class NodeT, class R>
__device__ __forceinline__ void force_velocity(const NodeT& nd, R phi, R gx, R gy, R gz, R lap, const DevParams& P,
                                               R& Fx, R& Fy, R& Fz, R& ux, R& uy, R& uz) {
    const R br = coef<R>(P).sw15 * (dwell_d(phi) * coef<R>(P).inv_W2 - lap);
    Fx = br * gx + phi * coef<R>(P).g[0];
    Fy = br * gy + phi * coef<R>(P).g[1];
    Fz = br * gz + phi * coef<R>(P).g[2];
    R jx, jy, jz;
    nd.flow_j(jx, jy, jz);
    ux = R(3) * jx + R(0.5) * Fx;
    uy = R(3) * jy + R(0.5) * Fy;
    uz = R(3) * jz + R(0.5) * Fz;
}

// reciprocal rounded to nearest (__frcp_rn), cheaper than a full FP32 division
__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }

// e . v for a lattice vector with components in {-1, 0, 1}, without multiplications
template <class R>
__device__ __forceinline__ R edot(int ex, int ey, int ez, R vx, R vy, R vz) {
    R s = R(0);
    if (ex) s = ex > 0 ? vx : -vx;
    if (ey) s = ey > 0 ? s + vy : s - vy;
    if (ez) s = ez > 0 ? s + vz : s - vz;
    return s;
}

// Collisions of one node (steps a6-a8) and the scatter of the post-collision values.
// Each BGK update keeps the form P* = P - om (P - P^eq) (+ source), which rounds only the
// small non-equilibrium difference; the equilibria reuse node-wide terms:
//   f:  Gamma_k = w (A + cu (3 + 4.5 cu)), A = 1 - 1.5 u^2; F_k = Gamma_k (e.F - u.F);
//       f^eq = w (B + cu (1 + 1.5 cu)) - F_k / 2, B = p_h - 0.5 u^2          (Eqs. 36-39)
//   g:  g^eq = w (phi - S/2 + phi cu / cs2), g* = g - om (g - g^eq) + w S    (Eqs. 46-48)
//   h:  h^eq_k = w (mu + c cu / cs2), h^eq_0 = dc - (1 - w_0) mu (shifted)   (Eqs. 50-51)
// With 16-bit storage the moving populations are updated per unit weight (Codec16Pop): every
// term above carries the factor w_k, so dividing it out leaves the same affine update with
// the per-direction weights gone, e.g. x*_f = x - om (x - E_k) + G_k with x = f_k / w_k,
// E_k = f^eq / w_k, G_k = F_k / w_k.
// COLL: flow collision fixed at compile time (0 BGK, 1 TRT, 2 MRT); -1 reads P.coll to
// choose between BGK and TRT only, -2 reads it to choose among all three.
// MRT on the D3Q19 moment basis: d = f - f^eq, dm_i = (rate_i / |M_i|^2) sum_k M_ik d_k,
// f*_k = f_k - sum_i M_ik dm_i + F_k (M^-1 = M^T diag(1 / |M_i|^2)).
// The basis rows are even or odd under k -> opp(k), so the transform runs on the pair sums
// s = d_a + d_opp(a) (even rows) and differences t = d_a - d_opp(a) (odd rows), and the
// back-transform gives r_a = E + O, r_opp(a) = E - O: about half the products of the dense
// 19 x 19 forms. put(0, r_0) comes first, then the pairs in order.
__host__ __device__ constexpr bool mrt_even_row_of_basis(int i) {
    for (int k = 1; k < 19; ++k)
        if (MRT19::m(i, k) != MRT19::m(i, opp(k))) return false;
    return true;
}
// even rows as a mask, so that the test folds to a constant in the unrolled loops (a loop
// evaluated per node would run the basis in FP64 at run time)
constexpr unsigned kMrtEvenRows = (1u << 0) | (1u << 1) | (1u << 2) | (1u << 9) | (1u << 10) | (1u << 11) |
                                  (1u << 12) | (1u << 13) | (1u << 14) | (1u << 15);
__host__ __device__ constexpr bool mrt_mask_matches_basis() {
    for (int i = 0; i < 19; ++i)
        if (mrt_even_row_of_basis(i) != bool((kMrtEvenRows >> i) & 1u)) return false;
    return true;
}
static_assert(mrt_mask_matches_basis(), "even/odd rows of the D3Q19 moment basis");
__host__ __device__ constexpr bool mrt_even_row(int i) { return (kMrtEvenRows >> i) & 1u; }
template <class R, class Pre, class Post>
__device__ __forceinline__ void mrt_relax(const DevParams& P, Pre d_of, Post put) {
    R d0 = d_of(0);
    R s[9], t[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const R a = d_of(2 * p + 1), b = d_of(2 * p + 2);
        s[p] = a + b;
        t[p] = a - b;
    }
    R dm[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        R acc = R(0);
        if (mrt_even_row(i)) {
            if (MRT19::m(i, 0) != 0.0) acc = R(MRT19::m(i, 0)) * d0;
#pragma unroll
            for (int p = 0; p < 9; ++p)
                if (MRT19::m(i, 2 * p + 1) != 0.0) acc += R(MRT19::m(i, 2 * p + 1)) * s[p];
        } else {
#pragma unroll
            for (int p = 0; p < 9; ++p)
                if (MRT19::m(i, 2 * p + 1) != 0.0) acc += R(MRT19::m(i, 2 * p + 1)) * t[p];
        }
        dm[i] = acc * coef<R>(P).mrt[i];
    }
    R r0 = R(0);
#pragma unroll
    for (int i = 0; i < 19; ++i)
        if (mrt_even_row(i) && MRT19::m(i, 0) != 0.0) r0 += R(MRT19::m(i, 0)) * dm[i];
    put(0, r0);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        R e = R(0), o = R(0);
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            if (MRT19::m(i, 2 * p + 1) == 0.0) continue;
            if (mrt_even_row(i)) e += R(MRT19::m(i, 2 * p + 1)) * dm[i];
            else o += R(MRT19::m(i, 2 * p + 1)) * dm[i];
        }
        put(2 * p + 1, e + o);
        put(2 * p + 2, e - o);
    }
}

template <class T, int LAT, bool FLOW, class A, int COLL = -2>
__device__ __forceinline__ void collide_store(const Node<T, LAT, FLOW>& nd, typename RealOf<T>::type phi,
                                              typename RealOf<T>::type ux, typename RealOf<T>::type uy,
                                              typename RealOf<T>::type uz, typename RealOf<T>::type Fx,
                                              typename RealOf<T>::type Fy, typename RealOf<T>::type Fz,
                                              const StateView& out, const A& ad, const DevParams& P) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    constexpr int Q = L::Q;
    const int self = ad.self;
    auto collide_f = [&]() {
        if constexpr (FLOW) {
            const R ph = nd.flow_p();
            const R usq = ux * ux + uy * uy + uz * uz;
            const R Ac = R(1) - R(1.5) * usq;
            const R Bc = ph - R(0.5) * usq;
            const R uF = ux * Fx + uy * Fy + uz * Fz;
            const R omf = coef<R>(P).om_f;
            // G = F_k / w_k (Eqs. 37-38) and E = f^eq_k / w_k (Eq. 39) of direction k
            auto force_eq = [&](int k, R& G, R& E) {
                const int ex = D3Q19::ex(k), ey = D3Q19::ey(k), ez = D3Q19::ez(k);
                const R cu = edot(ex, ey, ez, ux, uy, uz);
                G = (Ac + cu * (R(3) + R(4.5) * cu)) * (edot(ex, ey, ez, Fx, Fy, Fz) - uF);
                E = Bc + cu * (R(1) + R(1.5) * cu) - R(0.5) * G;
            };
            // the same for the opposite pair (k, k + 1): e.u and e.F change sign, so the even
            // parts (A + 4.5 cu^2, B + 1.5 cu^2) are shared (1 % faster for the D3Q7 fused kernel;
            // the per-node D3Q19 step, at 128 registers, keeps one direction at a time for BGK:
            // 7,519 against 6,507 MLUPS)
            auto force_eq_pair = [&](int k, R& Ga, R& Ea, R& Gb, R& Eb) {
                const int ex = D3Q19::ex(k), ey = D3Q19::ey(k), ez = D3Q19::ez(k);
                const R cu = edot(ex, ey, ez, ux, uy, uz);
                const R eF = edot(ex, ey, ez, Fx, Fy, Fz);
                const R c2 = cu * cu;
                const R Pe = Ac + R(4.5) * c2, Qe = Bc + R(1.5) * c2, t = R(3) * cu;
                Ga = (Pe + t) * (eF - uF);
                Gb = (t - Pe) * (eF + uF);
                Ea = Qe + cu - R(0.5) * Ga;
                Eb = Qe - cu - R(0.5) * Gb;
            };
            if constexpr (!is16<T>()) {
                auto put = [&](int k, R post) {
                    const Slot s = ad.dst(k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k));
                    *element<T, 0>(out, k, s) = post;
                };
                // F_k and f^eq_k in natural units
                auto force_eq_w = [&](int k, R& Fk, R& feq) {
                    const int ex = D3Q19::ex(k), ey = D3Q19::ey(k), ez = D3Q19::ez(k);
                    const R w = R(D3Q19::w(k));
                    const R cu = edot(ex, ey, ez, ux, uy, uz);
                    Fk = w * (Ac + cu * (R(3) + R(4.5) * cu)) * (edot(ex, ey, ez, Fx, Fy, Fz) - uF);
                    feq = w * (Bc + cu * (R(1) + R(1.5) * cu)) - R(0.5) * Fk;
                };
                const int coll = COLL >= 0 ? COLL : (COLL == -1 && P.coll == 2 ? 0 : P.coll);
                if (coll == 0 && Q == 19) {                       // BGK, Eq. 36 (see kPairs)
    #pragma unroll
                    for (int k = 0; k < 19; ++k) {
                        R Fk, feq;
                        force_eq_w(k, Fk, feq);
                        put(k, nd.f[k] - omf * (nd.f[k] - feq) + Fk);
                    }
                } else if (coll == 0) {                           // BGK, Eq. 36
                    R F0, feq0;
                    force_eq_w(0, F0, feq0);
                    put(0, nd.f[0] - omf * (nd.f[0] - feq0) + F0);
    #pragma unroll
                    for (int k = 1; k < 19; k += 2) {             // pairs (k, opp(k) = k + 1)
                        const R w = R(D3Q19::w(k));
                        R Ga, Ea, Gb, Eb;
                        force_eq_pair(k, Ga, Ea, Gb, Eb);
                        put(k, nd.f[k] - omf * (nd.f[k] - w * Ea) + w * Ga);
                        put(k + 1, nd.f[k + 1] - omf * (nd.f[k + 1] - w * Eb) + w * Gb);
                    }
                } else if ((COLL == 2 || COLL == -2) && coll == 2) {   // multiple relaxation times
                    R fF[19];                                  // f_k + F_k: f_k is dead after d_k
                    mrt_relax<R>(P, [&](int k) {
                        R Fk, feq;
                        force_eq_w(k, Fk, feq);
                        fF[k] = nd.f[k] + Fk;
                        return nd.f[k] - feq;
                    }, [&](int k, R r) { put(k, fF[k] - r); });
                } else {                                          // two relaxation times
                    const R omm = coef<R>(P).om_fm;
                    R F0, feq0;
                    force_eq_w(0, F0, feq0);
                    put(0, nd.f[0] - omf * (nd.f[0] - feq0) + F0);
    #pragma unroll
                    for (int k = 1; k < 19; k += 2) {             // pairs (k, opp(k) = k + 1)
                        const R w = R(D3Q19::w(k));
                        R Ga, Ea, Gb, Eb;
                        force_eq_pair(k, Ga, Ea, Gb, Eb);
                        const R Fa = w * Ga, Fb = w * Gb;
                        const R da = nd.f[k] - w * Ea, db = nd.f[k + 1] - w * Eb;
                        const R even = R(0.5) * (da + db), odd = R(0.5) * (da - db);
                        put(k, nd.f[k] - omf * even - omm * odd + Fa);
                        put(k + 1, nd.f[k + 1] - omf * even + omm * odd + Fb);
                    }
                }
            } else {
                // 16-bit storage: nd.f[k] = f_k / w_k for k > 0 (the writer's reference added back
                // on load), nd.f[0] = f_0. The updates below are those of the FP32 branch divided by
                // w_k. f*_0 is stored first, in FP32, and is the reference of every moving
                // population this node stores: x*_k - f*_0 / w_0 is what gets rounded.
                using C = Codec<T>;
                constexpr float u = C::template unit<SET_F>();
                R nref = R(0);                                    // -u f*_0 / w_0
                auto put0 = [&](R f0post) {
                    const float f0s = float(f0post);
                    out.rest[A::kF0Out * P.plane + self] = f0s;
                    nref = R(f0s) * R(-u / D3Q19::w(0));
                };
                auto put = [&](int k, R x) {                      // x = f*_k / w_k
                    const Slot sl = ad.dst(k, D3Q19::ex(k), D3Q19::ey(k), D3Q19::ez(k));
                    *element<T, 0>(out, k, sl) = C::template enc<SET_F>(fmaf(float(x), u, float(nref)));
                };
                const R w0 = R(D3Q19::w(0));
                const int coll = COLL >= 0 ? COLL : (COLL == -1 && P.coll == 2 ? 0 : P.coll);
                if ((COLL == 2 || COLL == -2) && coll == 2) {
                    // MRT mixes directions: run it on the populations in natural units
                    R fF[19];                                  // per unit weight, f_k / w_k + G_k
                    mrt_relax<R>(P, [&](int k) {
                        R G, E;
                        force_eq(k, G, E);
                        const R w = R(D3Q19::w(k));
                        if (k == 0) {
                            fF[0] = nd.f[0] + w * G;
                            return nd.f[0] - w * E;
                        }
                        fF[k] = nd.f[k] + G;
                        return w * (nd.f[k] - E);
                    }, [&](int k, R r) {
                        if (k == 0) put0(fF[0] - r);
                        else put(k, fF[k] - r * R(1.0 / D3Q19::w(k)));
                    });
                } else {
                    R G0, E0;
                    force_eq(0, G0, E0);
                    put0(nd.f[0] - omf * (nd.f[0] - w0 * E0) + w0 * G0);
                    if (coll == 0) {
    #pragma unroll
                        for (int k = 1; k < 19; k += 2) {
                            R Ga, Ea, Gb, Eb;
                            force_eq_pair(k, Ga, Ea, Gb, Eb);
                            put(k, nd.f[k] - omf * (nd.f[k] - Ea) + Ga);
                            put(k + 1, nd.f[k + 1] - omf * (nd.f[k + 1] - Eb) + Gb);
                        }
                    } else {
                        const R omm = coef<R>(P).om_fm;
    #pragma unroll
                        for (int k = 1; k < 19; k += 2) {
                            R Ga, Ea, Gb, Eb;
                            force_eq_pair(k, Ga, Ea, Gb, Eb);
                            const R da = nd.f[k] - Ea, db = nd.f[k + 1] - Eb;
                            const R even = R(0.5) * (da + db), odd = R(0.5) * (da - db);
                            put(k, nd.f[k] - omf * even - omm * odd + Ga);
                            put(k + 1, nd.f[k + 1] - omf * even + omm * odd + Gb);
                        }
                    }
                }
            }
        }
    };
    auto collide_s = [&]() {
        const R p = interp_p(phi);
        const R muA = closure_dev(nd.dcA, p, 0, P);
        const R muB = closure_dev(nd.dcB, p, 1, P);
        const R inv_cs2 = R(1.0 / L::cs2());
        const R omg = coef<R>(P).om_g;
        const R MA = coef<R>(P).M0[0] * (R(1) - phi) + coef<R>(P).M1[0] * phi;     // §2.3
        const R MB = coef<R>(P).M0[1] * (R(1) - phi) + coef<R>(P).M1[1] * phi;
        const R omA = recip(MA * inv_cs2 + R(0.5));                      // tau_h = M / c_s^2
        const R omB = recip(MB * inv_cs2 + R(0.5));
        const R ga = phi - R(0.5) * nd.S;                                 // g^eq = w (ga + gb cu)
        const R gb = phi * inv_cs2;
        const R cAu = nd.cA(P) * inv_cs2, cBu = nd.cB(P) * inv_cs2;
        // rest populations (natural units in every storage), stored last
        R g0, hA0, hB0;
        if constexpr (!is16<T>()) {
            // The collisions keep sum g = phi~ + S and sum h = c - c_0^eq at the node (Eqs.
            // 47-48, 51 with the shifted h_0): each rest population takes that total minus the
            // moving populations it stores. Rounding the 2 Q collided values independently
            // instead leaves a node's sums off by a few units in the last place, the same at
            // every node of a uniform region, which adds up to a drift of the lattice totals.
            g0 = phi + R(0.5) * nd.S;                                     // phi~ + S
            hA0 = nd.dcA;
            hB0 = nd.dcB;
    #pragma unroll
            for (int k = 1; k < Q; ++k) {
                const int ex = L::ex(k), ey = L::ey(k), ez = L::ez(k);
                const R w = R(L::w(k));
                const R cu = edot(ex, ey, ez, ux, uy, uz);
                const R geq = w * (ga + gb * cu);
                const R gpost = nd.g[k] - omg * (nd.g[k] - geq) + w * nd.S;
                const R hApost = nd.hA[k] - omA * (nd.hA[k] - w * (muA + cAu * cu));
                const R hBpost = nd.hB[k] - omB * (nd.hB[k] - w * (muB + cBu * cu));
                const Slot s = ad.dst(k, ex, ey, ez);
                *element<T, Planes<LAT>::G>(out, k, s) = gpost;
                *element<T, Planes<LAT>::HA>(out, k, s) = hApost;
                *element<T, Planes<LAT>::HB>(out, k, s) = hBpost;
                g0 -= gpost;
                hA0 -= hApost;
                hB0 -= hBpost;
            }
        } else {
            // the collisions keep sum g = phi~ + S and sum h = c - c_0^eq (Eqs. 47-48, 51 with the
            // shifted h_0); each rest population takes that total minus what the moving ones stored
            g0 = phi + R(0.5) * nd.S - R(0.5 * (1.0 - L::w(0)));       // phi~ + S = phi + S/2
            hA0 = nd.dcA;
            hB0 = nd.dcB;
            // in storage units r = u x: g = w (x + 1/2) (u = 1) gives x* = x - om (x + 1/2 - ga -
            // gb cu) + S, and h = (w / u) r gives r* = r - om (r - u (mu + c cu / cs2))
            using C = Codec<T>;
            static_assert(C::template unit<SET_G>() == 1.0f, "g in units of x");
            constexpr float uh = C::template unit<SET_H>();
            const R gq = R(0.5) - ga;
            const R mA = R(uh) * muA, mB = R(uh) * muB;
            const R cA = R(uh) * cAu, cB = R(uh) * cBu;
    #pragma unroll
            for (int k = 1; k < Q; ++k) {
                const int ex = L::ex(k), ey = L::ey(k), ez = L::ez(k);
                const R cu = edot(ex, ey, ez, ux, uy, uz);
                const Slot s = ad.dst(k, ex, ey, ez);
                const R qg = nd.g[k] - omg * (nd.g[k] + gq - gb * cu) + nd.S;
                const R qA = nd.hA[k] - omA * (nd.hA[k] - (mA + cA * cu));
                const R qB = nd.hB[k] - omB * (nd.hB[k] - (mB + cB * cu));
                g0 -= R(C::template scale<SET_G>(L::w(k))) *
                      C::template store_back<SET_G>(element<T, Planes<LAT>::G>(out, k, s), qg);
                hA0 -= R(C::template scale<SET_H>(L::w(k))) *
                       C::template store_back<SET_H>(element<T, Planes<LAT>::HA>(out, k, s), qA);
                hB0 -= R(C::template scale<SET_H>(L::w(k))) *
                       C::template store_back<SET_H>(element<T, Planes<LAT>::HB>(out, k, s), qB);
            }
        }
        const Slot s0{self, 0};
        store_scalar<T, SET_G, LAT, Planes<LAT>::G, 0>(out, 0, s0, g0, P);
        store_scalar<T, SET_H, LAT, Planes<LAT>::HA, 1>(out, 0, s0, hA0, P);
        store_scalar<T, SET_H, LAT, Planes<LAT>::HB, 2>(out, 0, s0, hB0, P);
    };
    // D3Q7 scalar sets first: their populations are dead before the flow collision needs the
    // registers (MRT: no spills; BGK with the compensated rest populations: 16,193 MLUPS at
    // 512^3 against 14,798 with the flow collision first). The 57 populations of D3Q19 scalar
    // sets go after the flow's 19 (the per-node D3Q19 step ran at 6,037 against 7,783 MLUPS
    // the other way round).
    if constexpr (Q == 19) {
        collide_f();
        collide_s();
    } else {
        collide_s();
        collide_f();
    }
}

// ------------------------------------------------------------------------------------
// One coupled step per node. With flow the phi field of this step must already be in
// phi_field (phi pass); MODE AA_* works in place on ``st``, PULL reads ``st`` and writes ``out``.
template <class T, int LAT, bool FLOW, int MODE, int COLL>
__global__ void __launch_bounds__(kBlockX)
step_kernel(const DevParams P, const StateView st, const StateView out,
            const typename RealOf<T>::type* __restrict__ phi_field) {
    using R = typename RealOf<T>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + P.z_lo;
    if (x >= P.nx) return;
    Addr<MODE> ad;
    ad.self = node_of(x, y, z, P);
    ad.nb.init(x, y, z, P);
    Node<T, LAT, FLOW> nd;
    nd.gather(st, ad, P);
    nd.moments(P);
    R phi;
    if constexpr (FLOW) phi = phi_field[ad.self]; else phi = nd.phi();
    R ux = R(0), uy = R(0), uz = R(0), Fx = R(0), Fy = R(0), Fz = R(0);
    if constexpr (FLOW) {
        R gx, gy, gz, lap;
        stencil([&](int dx, int dy, int dz) { return ad.phi(phi_field, dx, dy, dz); }, phi, gx, gy, gz, lap);
        force_velocity(nd, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
    }
    collide_store<T, LAT, FLOW, Addr<MODE>, COLL>(nd, phi, ux, uy, uz, Fx, Fy, Fz, out, ad, P);
}

// phi = sum g + S/2 of every node (Eq. 49), read by the capillary stencil.
template <class T, int LAT, int MODE>
__global__ void __launch_bounds__(kBlockX)
phi_kernel(const DevParams P, const StateView st, typename RealOf<T>::type* __restrict__ phi_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + P.z_lo;
    if (x >= P.nx) return;
    Addr<MODE> ad;
    ad.self = node_of(x, y, z, P);
    ad.nb.init(x, y, z, P);
    Node<T, LAT, false> nd;
    nd.gather_scalars(st, ad, P);
    nd.moments(P);
    phi_out[ad.self] = nd.phi();
}

// phi (Eq. 49) of plane z into out[y nx + x]: a slab's edge plane, sent to the neighbouring
// slab whose capillary stencil reads it (the same arithmetic as phi_kernel and the fused
// kernel's ring, so a slab run matches the undivided lattice bit for bit).
template <class T, int LAT, int MODE>
__global__ void __launch_bounds__(kBlockX)
plane_phi_kernel(const DevParams P, const StateView st, int z, typename RealOf<T>::type* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= P.nx) return;
    Addr<MODE> ad;
    ad.self = node_of(x, y, z, P);
    ad.nb.init(x, y, z, P);
    Node<T, LAT, false> nd;
    nd.gather_scalars(st, ad, P);
    nd.moments(P);
    out[y * P.nx + x] = nd.phi();
}

// ------------------------------------------------------------------------------------
// Fused two-buffer flow step: each CTA marches an (FX x FY) column of (x, y) through a
// chunk of z planes. At each plane z:
//   fill(z + 1): every thread gathers the scalar populations (g, h^A, h^B) of its own
//     column at plane z + 1, keeps them decoded in shared memory (double-buffered) with
//     S (and c - c_0^eq with 16-bit storage), and writes phi into a 4-plane ring; 84
//     threads add the ring's one-node halo.
//   centre(z): gather the 19 f populations, take the scalar populations of plane z from
//     shared memory, form the capillary stencil from the ring, collide and store f, then
//     collide and store g, h^A, h^B (all stores local and coalesced).
// The ring holds four planes, so one barrier per plane suffices: fill(z + 2) overwrites the
// plane of z - 2, which no thread can still be reading once all have passed the barrier
// after fill(z + 1). The stencil therefore needs no separate pass and the scalar
// populations are read from HBM once; the halo re-reads hit L2.
constexpr int FX = 32, FY = 8, FT = FX * FY;
constexpr int kHalo = 2 * (FX + 2) + 2 * FY;    // ring positions outside the tile (84)
// Parked per tile node: 21 scalar populations and S, plus c - c_0^eq with 16-bit storage.
// FP32/FP64 sum c - c_0^eq again from the parked h instead: the 4 KB saved per block let
// three blocks fit the 164 KB shared-memory carveout, leaving 92 KB of L1 rather than 60 KB
// for the gathers in flight (1.4 % faster); the instruction-bound 16-bit kernel parks it
// (6 % faster than summing it again).
template <class T> constexpr bool park_dc() { return is16<T>(); }
template <class T> constexpr int spops_n() { return 3 * 7 + (park_dc<T>() ? 3 : 1); }

// With 16-bit storage a second ring holds the FP32 f_0 of the same positions: the reference
// of the populations each node stored (Codec16Pop), read by the 18 nodes that pull them.
template <class T>
__host__ __device__ constexpr size_t fused_smem_bytes() {
    using R = typename RealOf<T>::type;
    return sizeof(R) * (4 * (FY + 2) * (FX + 2) + 2 * spops_n<T>() * FT) +
           (is16<T>() ? sizeof(float) * 4 * (FY + 2) * (FX + 2) : 0);
}

// COLL: the flow collision of this instance. FP32/FP64 storage keeps BGK and TRT in one
// instance behind a block-uniform branch on P.coll (measured 1 % faster for BGK than a
// BGK-only instance at this register budget); 16-bit storage and MRT get instances of their
// own (the 16-bit BGK instance is 6 % faster without the TRT code).
// SLAB: the lattice is a slab of a z decomposition (planes [z_lo, z_hi), ghost planes
// beyond); the undivided lattice takes an instance without that code.
// Blocks per SM the register budget is cut for: three (80 registers). (MRT at two blocks and
// 128 registers, without spills, measured 8 % slower than three blocks with a few spills.)
template <class T, int COLL>
constexpr int fused_min_blocks() { return sizeof(typename RealOf<T>::type) == 8 ? 1 : 3; }

template <class T, int COLL, bool SLAB>
__global__ void __launch_bounds__(FT, fused_min_blocks<T, COLL>())
fused_flow_kernel(const DevParams P, const StateView src, const StateView dst, int zchunk) {
    constexpr int kColl = (!is16<T>() && COLL != 2) ? -1 : COLL;
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT_D3Q7>;
    constexpr int Q = L::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R (*ring)[FY + 2][FX + 2] = reinterpret_cast<R (*)[FY + 2][FX + 2]>(smem_raw);
    R* spops = reinterpret_cast<R*>(smem_raw) + 4 * (FY + 2) * (FX + 2);   // [2][spops_n][FT]
    constexpr int kSPops = spops_n<T>();
    // f_0 / w_0 of the ring's positions (16-bit storage)
    float (*fring)[FY + 2][FX + 2] = reinterpret_cast<float (*)[FY + 2][FX + 2]>(spops + 2 * kSPops * FT);
    constexpr float kInvW0 = float(1.0 / D3Q19::w(0));
    constexpr bool kParkDc = park_dc<T>();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * FX + tx;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * FY;
    const int zs = SLAB ? P.z_lo + blockIdx.z * zchunk : blockIdx.z * zchunk;
    const int ze = min(zs + zchunk, SLAB ? P.z_hi : P.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < P.nx && y < P.ny;

    // domain column of ring position (hx, hy): periodic wrap in x and y, mirror across x walls
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
        if (zz < 0) return (SLAB ? P.wall_zlo : P.wall_z) ? 0 : zz + P.nz;
        if (zz >= P.nz) return (SLAB ? P.wall_zhi : P.wall_z) ? P.nz - 1 : zz - P.nz;
        return zz;
    };
    // this thread's own ring column and its halo column (threads tid < kHalo), fixed in z
    int ox, oy, hxp = 0, hyp = 0, hgx = 0, hgy = 0;
    const bool own_ok = wrap_xy(tx, ty, ox, oy);
    bool halo_ok = false;
    if (tid < kHalo) {
        if (tid < FX + 2) { hxp = tid - 1; hyp = -1; }
        else if (tid < 2 * (FX + 2)) { hxp = tid - (FX + 2) - 1; hyp = FY; }
        else if (tid < 2 * (FX + 2) + FY) { hxp = -1; hyp = tid - 2 * (FX + 2); }
        else { hxp = FX; hyp = tid - 2 * (FX + 2) - FY; }
        halo_ok = wrap_xy(hxp, hyp, hgx, hgy);
    }
    Addr<PULL> own, halo;
    own.nb.init_xy(ox, oy, P);
    halo.nb.init_xy(hgx, hgy, P);
    // blocks whose ring (tile + one-node halo) and its pull sources stay inside the lattice
    // in x and y take the AddrInterior path on every plane z with 1 <= z <= nz - 2: one
    // branch per plane, uniform across the block
    const bool xy_inner = x0 >= 2 && x0 + FX + 2 <= P.nx && y0 >= 2 && y0 + FY + 2 <= P.ny;
    const int sxy = P.nx * P.ny;
    auto inner_plane = [&](int zr) { return xy_inner && zr >= 1 && zr <= P.nz - 2; };

    // phi (and, for a tile node, its scalar populations in buffer buf) of plane zz
    auto fill = [&](auto fast, int zz, int s, int buf) {
        constexpr bool kFast = decltype(fast)::value;
        const int zr = zwrap(zz);
        R v = R(0);
        if (own_ok) {
            Node<T, LAT_D3Q7, false> nd;
            if constexpr (kFast) {
                nd.gather_scalars(src, AddrInterior{node_of(ox, oy, zr, P), P.nx, sxy}, P);
            } else {
                own.self = node_of(ox, oy, zr, P);
                own.nb.set_z(zr, P);
                nd.gather_scalars(src, own, P);
            }
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
                if constexpr (kParkDc) {
                    sp[(3 * Q + 1) * FT] = nd.dcA;
                    sp[(3 * Q + 2) * FT] = nd.dcB;
                }
            }
        }
        ring[s][ty + 1][tx + 1] = v;
        if constexpr (is16<T>())
            fring[s][ty + 1][tx + 1] = own_ok ? src.rest[3 * P.plane + node_of(ox, oy, zr, P)] * kInvW0 : 0.f;
        if (tid < kHalo) {
            R hv = R(0);
            if (halo_ok) {
                Node<T, LAT_D3Q7, false> nd;
                if constexpr (kFast) {
                    nd.gather_scalars(src, AddrInterior{node_of(hgx, hgy, zr, P), P.nx, sxy}, P);
                } else {
                    halo.self = node_of(hgx, hgy, zr, P);
                    halo.nb.set_z(zr, P);
                    nd.gather_scalars(src, halo, P);
                }
                nd.moments(P);
                hv = nd.phi();
            }
            ring[s][hyp + 1][hxp + 1] = hv;
            if constexpr (is16<T>())
                fring[s][hyp + 1][hxp + 1] = halo_ok ? src.rest[3 * P.plane + node_of(hgx, hgy, zr, P)] * kInvW0 : 0.f;
        }
    };

    using Fast = std::true_type;
    using Slow = std::false_type;
    // a slab's neighbouring planes (z_lo - 1, z_hi): their phi arrives from the neighbour
    // (phi_ghost), with 16-bit storage their f_0 with the populations
    auto fill_ghost = [&](const R* gh, int zz, int s) {
        ring[s][ty + 1][tx + 1] = own_ok ? gh[oy * P.nx + ox] : R(0);
        if (tid < kHalo) ring[s][hyp + 1][hxp + 1] = halo_ok ? gh[hgy * P.nx + hgx] : R(0);
        if constexpr (is16<T>()) {
            const float* f0 = src.rest + 3 * P.plane;
            fring[s][ty + 1][tx + 1] = own_ok ? f0[node_of(ox, oy, zz, P)] * kInvW0 : 0.f;
            if (tid < kHalo) fring[s][hyp + 1][hxp + 1] = halo_ok ? f0[node_of(hgx, hgy, zz, P)] * kInvW0 : 0.f;
        }
    };
    auto fill_any = [&](int zz, int s, int buf) {
        if constexpr (SLAB) {
            if (zz < P.z_lo && P.phi_ghost[0]) { fill_ghost(static_cast<const R*>(P.phi_ghost[0]), zz, s); return; }
            if (zz >= P.z_hi && P.phi_ghost[1]) { fill_ghost(static_cast<const R*>(P.phi_ghost[1]), zz, s); return; }
        }
        if (inner_plane(zwrap(zz))) fill(Fast{}, zz, s, buf);
        else fill(Slow{}, zz, s, buf);
    };
    // centre(z) of an active thread, with either addressing
    auto centre = [&](const auto& ad, int z) {
        const int sp = (z - 1) & 3, sc = z & 3, sn = (z + 1) & 3;
        Node<T, LAT_D3Q7, true> nd;
        // 16-bit storage: the writers' f_0 / w_0 from the ring (the node itself across a wall)
        nd.gather_flow(src, ad, P, [&](int k, int ex, int ey, int ez, Slot s) {
            if (k == 0 || s.node == ad.self) return fring[sc][ty + 1][tx + 1];
            return fring[ez > 0 ? sp : (ez < 0 ? sn : sc)][ty + 1 - ey][tx + 1 - ex];
        });
        const R* spc = spops + (z & 1) * kSPops * FT + tid;
        nd.S = spc[(3 * Q) * FT];
        if constexpr (kParkDc) {
            nd.dcA = spc[(3 * Q + 1) * FT];
            nd.dcB = spc[(3 * Q + 2) * FT];
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            nd.g[k] = spc[k * FT];
            nd.hA[k] = spc[(Q + k) * FT];
            nd.hB[k] = spc[(2 * Q + k) * FT];
        }
        if constexpr (!kParkDc) nd.dc_sums();
        const R phi = ring[sc][ty + 1][tx + 1];
        R gx, gy, gz, lap, Fx, Fy, Fz, ux, uy, uz;
        stencil([&](int dx, int dy, int dz) {
                    const int s = dz < 0 ? sp : (dz > 0 ? sn : sc);
                    return ring[s][ty + 1 + dy][tx + 1 + dx];
                }, phi, gx, gy, gz, lap);
        force_velocity(nd, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
        collide_store<T, LAT_D3Q7, true, std::decay_t<decltype(ad)>, kColl>(nd, phi, ux, uy, uz, Fx, Fy, Fz, dst,
                                                                            ad, P);
    };

    fill_any(zs - 1, (zs - 1) & 3, -1);
    fill_any(zs, zs & 3, zs & 1);
    for (int z = zs; z < ze; ++z) {
        fill_any(z + 1, (z + 1) & 3, (z + 1) & 1);
        __syncthreads();
        if (active) {
            if (inner_plane(z)) {
                centre(AddrInterior{node_of(x, y, z, P), P.nx, sxy}, z);
            } else {
                own.self = node_of(x, y, z, P);
                own.nb.set_z(z, P);
                centre(own, z);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Initial populations at rest (Eqs. 47, 51 and 37-39 at u = 0, p_h = 0), in the storage's
// arithmetic type (FP32 for FP32 and 16-bit storage, like every later step; GB300's FP64 pipe
// would make this kernel several steps long). The FP64 inputs are read once and the
// compositions shifted by c_0^eq in FP64 before the conversion, so the closure's cancellation
// starts from the exact deviations. Each node evaluates its phi_0-derived quantities once and
// stores its population k in the slot its own first gather of k will read (Addr<MODE>::src):
// its own slot k for AA_EVEN; for PULL slot k of node x - e_k, or, when that lies beyond a
// wall, its own slot opp(k). Every slot has exactly one writer.
template <class T, int LAT, bool FLOW, int MODE>
__global__ void __launch_bounds__(kBlockX)
init_kernel(const DevParams P, const StateView st, const double* __restrict__ phi0,
            const double* __restrict__ cA0, const double* __restrict__ cB0) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + P.z_lo;
    if (x >= P.nx) return;
    Addr<MODE> ad;
    ad.self = node_of(x, y, z, P);
    ad.nb.init(x, y, z, P);
    const R ph = R(phi0[ad.self]);
    const R pp = interp_p(ph);
    const R dA = R(cA0[ad.self] - P.c0[0]), dB = R(cB0[ad.self] - P.c0[1]);
    const R muA = closure_dev(dA, pp, 0, P), muB = closure_dev(dB, pp, 1, P);
    const R S = source(ph, muA, muB, P);
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const R w = R(L::w(k));
        const Slot s = ad.src(k, L::ex(k), L::ey(k), L::ez(k));
        store_scalar<T, SET_G, LAT, Planes<LAT>::G, 0>(st, k, s, w * ph - R(0.5) * w * S, P);   // Eq. 47
        const R hA = k == 0 ? dA - (R(1) - w) * muA : w * muA;                               // Eq. 51,
        const R hB = k == 0 ? dB - (R(1) - w) * muB : w * muB;                               // h_0 shifted
        store_scalar<T, SET_H, LAT, Planes<LAT>::HA, 1>(st, k, s, hA, P);
        store_scalar<T, SET_H, LAT, Planes<LAT>::HB, 2>(st, k, s, hB, P);
    }
    if constexpr (FLOW) {
        R gx, gy, gz, lap;
        stencil([&](int dx, int dy, int dz) { return R(ad.phi(phi0, dx, dy, dz)); }, ph, gx, gy, gz, lap);
        const R br = coef<R>(P).sw15 * (dwell_d(ph) * coef<R>(P).inv_W2 - lap);
        const R Fx = br * gx + ph * coef<R>(P).g[0], Fy = br * gy + ph * coef<R>(P).g[1];
        const R Fz = br * gz + ph * coef<R>(P).g[2];
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const int ex = D3Q19::ex(k), ey = D3Q19::ey(k), ez = D3Q19::ez(k);
            const R v = R(-0.5 * D3Q19::w(k)) * edot(ex, ey, ez, Fx, Fy, Fz);                // Eqs. 37-39
            const Slot s = ad.src(k, ex, ey, ez);
            if (is16<T>() && k == 0) st.rest[3 * P.plane + s.node] = float(v);
            else Codec<T>::template store<SET_F>(element<T, 0>(st, k, s), v, D3Q19::w(k), P);
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
    const int y = blockIdx.y, z = blockIdx.z + P.z_lo;
    if (x >= P.nx) return;
    Addr<MODE> ad;
    ad.self = node_of(x, y, z, P);
    ad.nb.init(x, y, z, P);
    Node<T, LAT, FLOW> nd;
    nd.gather(st, ad, P);
    nd.moments(P);
    R phi;
    if constexpr (FLOW) phi = phi_field[ad.self]; else phi = nd.phi();
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
        force_velocity(nd, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, vals[6], vals[7], vals[8]);
        vals[5] = nd.flow_p();
    }
#pragma unroll
    for (int i = 0; i < LBM_NFIELDS_DEV; ++i)
        if (out.p[i]) static_cast<R*>(out.p[i])[ad.self] = vals[i];
}

template <int LAT> constexpr bool kTwoD = LAT == LAT_D2Q5 || LAT == LAT_D2Q9;

// Euler characteristic of the 8-connected set {phi >= 1/2} of a 2D lattice by Gray's bit
// quads: over all 2x2 windows, chi = (n1 - n3 - 2 nd) / 4 with n1 (n3) the windows holding
// one (three) set pixels and nd those holding a diagonal pair. Node (x, y) owns the window
// spanning x..x+1, y..y+1 (periodic wrap; outside an x wall counts as empty, and the node
// at x = 0 also owns the window reaching out to x = -1). Returns 4 times its share of chi.
template <class R>
__device__ __forceinline__ int euler_quads4(const R* __restrict__ phi, int x, int y, const DevParams& P) {
    const int yp = y + 1 < P.ny ? y + 1 : 0;
    auto on = [&](int xx, int yy) {
        return xx >= 0 && xx < P.nx && phi[yy * P.nx + xx] >= R(0.5);
    };
    auto window = [&](int x0, int x1) {
        const int a = on(x0, y), b = on(x1, y), c = on(x0, yp), d = on(x1, yp);
        const int n = a + b + c + d;
        const int diag = (n == 2 && a == d) ? 1 : 0;
        return int(n == 1) - int(n == 3) - 2 * diag;
    };
    const int xp = x + 1 < P.nx ? x + 1 : (P.wall_x ? P.nx : 0);
    int q = window(x, xp);
    if (P.wall_x && x == 0) q += window(-1, 0);
    return q;
}

// Euler characteristic of the 26-connected set {phi >= 1/2} of a 3D lattice: the alternating
// count of the vertices, edges, faces and cubes of the union of closed unit cubes centred on
// the set nodes. Position (x, y, z) owns the cube of node (x, y, z), the faces on its low
// x, y and z sides, the edges along x, y and z through the corner line on its low sides, and
// its low corner vertex (x - 1/2, y - 1/2, z - 1/2); a cell belongs to the union when any
// node it bounds is set (b[c][b][a]: node (x - 1 + a, y - 1 + b, z - 1 + c)). Outside an x
// or z wall is empty; other axes wrap. bits: bit (id & 31) of word id >> 5 is node id's
// phi >= 1/2, ids x fastest.
__device__ __forceinline__ int euler_cells(const unsigned* __restrict__ bits, int x, int y, int z,
                                           const DevParams& P) {
    int b[2][2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                int xx = x - 1 + a, yy = y - 1 + bb, zz = z - 1 + c;
                bool inside = true;
                if (xx < 0) { inside = !P.wall_x; xx += P.nx; }
                if (xx >= P.nx) { inside = !P.wall_x; xx -= P.nx; }
                if (yy < 0) yy += P.ny;
                if (zz < 0) { inside = inside && !P.wall_z; zz += P.nz; }
                if (zz >= P.nz) { inside = inside && !P.wall_z; zz -= P.nz; }
                const unsigned id = (unsigned(zz) * unsigned(P.ny) + unsigned(yy)) * unsigned(P.nx) + unsigned(xx);
                b[c][bb][a] = inside ? int((__ldg(bits + (id >> 5)) >> (id & 31)) & 1u) : 0;
            }
    const int vert = b[0][0][0] | b[0][0][1] | b[0][1][0] | b[0][1][1] | b[1][0][0] | b[1][0][1] | b[1][1][0] |
                     b[1][1][1];
    const int ex = b[0][0][1] | b[0][1][1] | b[1][0][1] | b[1][1][1];
    const int ey = b[0][1][0] | b[0][1][1] | b[1][1][0] | b[1][1][1];
    const int ez = b[1][0][0] | b[1][0][1] | b[1][1][0] | b[1][1][1];
    const int fx = b[1][1][0] | b[1][1][1];
    const int fy = b[1][0][1] | b[1][1][1];
    const int fz = b[0][1][1] | b[1][1][1];
    return vert - (ex + ey + ez) + (fx + fy + fz) - b[1][1][1];
}

// Writes slot LBM_RED_EULER of every block's partials (the reduction kernel leaves it 0 on
// 3D lattices). Along a walled axis the cell positions run one past the last node: that
// node owns the positions on the wall too.
template <class T>
__global__ void __launch_bounds__(256)
euler3d_kernel(const DevParams P, const unsigned* __restrict__ bits, double* __restrict__ partials) {
    long long acc = 0;
    const unsigned stride = gridDim.x * blockDim.x;
    const unsigned nxy = unsigned(P.nx) * unsigned(P.ny), n = unsigned(P.n);
    for (unsigned id = blockIdx.x * blockDim.x + threadIdx.x; id < n; id += stride) {
        const unsigned zu = id / nxy, xy = id - zu * nxy;
        const unsigned yu = xy / unsigned(P.nx);
        const int x = int(xy - yu * unsigned(P.nx)), y = int(yu), z = int(zu);
        const int x1 = (P.wall_x && x == P.nx - 1) ? P.nx : x;
        const int z1 = (P.wall_z && z == P.nz - 1) ? P.nz : z;
        for (int zs = z; zs <= z1; ++zs)
            for (int xs = x; xs <= x1; ++xs) acc += euler_cells(bits, xs, y, zs, P);
    }
    __shared__ long long sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) sm[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        long long v = lane < int(blockDim.x >> 5) ? sm[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) partials[(long long)blockIdx.x * LBM_NRED_DEV + (LBM_NRED_DEV - 1)] = double(v);
    }
}

// Running sum of one thread in the reduction. FP64 storage sums in FP64. With FP32 arithmetic
// the sum is kept as an unevaluated pair hi + lo of FP32 numbers (float-float addition):
// TwoSum (Knuth, TAOCP vol. 2, §4.2.2) gives the exact rounding error e of hi + v, e joins lo,
// and FastTwoSum (Dekker 1971) renormalises the pair so that |lo| stays below half an ulp of
// hi. Each addition then errs by at most about 2^-47 of the running sum, n terms by n 2^-47
// (below 1e-11 relative for the ~1,200 nodes per thread of a 512^3 lattice), so the sums keep
// FP64-level accuracy while the per-node work stays on the FP32 pipes (this part's FP64 rate
// is a small fraction of its FP32 rate).
template <class R> struct SumAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct SumAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float s = hi + v;
        const float bv = s - hi;
        const float e = (hi - (s - bv)) + (v - bv);
        const float t = lo + e;
        hi = s + t;
        lo = t - (hi - s);
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// FP64 block partials of the global diagnostics (grid-stride over nodes; the 32 nodes a warp
// visits together are consecutive and start at a multiple of 32). On 3D lattices it also
// writes the bit field of phi >= 1/2 that euler3d_kernel reads, one warp vote per word.
// Node indices are 32-bit (the host rejects lattices of 2^31 nodes or more). Per-node values
// are formed in the kernels' arithmetic type and summed per thread (SumAcc); the c sums add
// c_0^eq once per node counted, and the thread and block totals are combined in FP64.
// blocks per SM the reduction's register budget is cut for: three (80 registers) with FP32
// arithmetic, two (128) for FP64 values or the 57 scalar populations of D3Q19
template <class T, int LAT> constexpr int reduce_min_blocks() {
    return (LAT == LAT_D3Q19 || sizeof(typename RealOf<T>::type) == 8) ? 2 : 3;
}

template <class T, int LAT, bool FLOW, int MODE>
__global__ void __launch_bounds__(256, (reduce_min_blocks<T, LAT>()))
reduce_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ phi_field,
              unsigned* __restrict__ bits, double* __restrict__ partials) {
    using R = typename RealOf<T>::type;
    SumAcc<R> s_phi, s_dcA, s_dcB, s_p, s_S, s_phit, s_int;
    R umax = R(0);
    int nodes = 0, bad = 0, quads = 0;
    const R kint = R(4.0 / P.W);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nxy = unsigned(P.nx) * unsigned(P.ny);
    const unsigned stride = gridDim.x * blockDim.x;
    // nodes of the planes [z_lo, z_hi); the bit field (3D Euler count) only when they start at 0
    const unsigned id0 = unsigned(P.z_lo) * nxy, id1 = unsigned(P.z_hi) * nxy;
    for (unsigned base = id0 + blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < id1; base += stride) {
        const unsigned id = base + lane;
        bool on = false;
        if (id < id1) {
            const unsigned z = id / nxy, xy = id - z * nxy;
            const unsigned y = xy / unsigned(P.nx), x = xy - y * unsigned(P.nx);
            Addr<MODE> ad;
            ad.self = int(id);
            ad.nb.init(int(x), int(y), int(z), P);
            Node<T, LAT, FLOW> nd;
            nd.gather(st, ad, P);
            nd.moments(P);
            R phi;
            if constexpr (FLOW) phi = phi_field[id]; else phi = nd.phi();
            R umag = R(0), ph = R(0);
            if constexpr (FLOW) {
                R gx, gy, gz, lap, Fx, Fy, Fz, ux, uy, uz;
                stencil([&](int dx, int dy, int dz) { return ad.phi(phi_field, dx, dy, dz); }, phi, gx, gy, gz, lap);
                force_velocity(nd, phi, gx, gy, gz, lap, P, Fx, Fy, Fz, ux, uy, uz);
                umag = sqrt(ux * ux + uy * uy + uz * uz);
                ph = nd.flow_p();
            }
            s_phi.add(phi);
            s_dcA.add(nd.dcA);
            s_dcB.add(nd.dcB);
            s_p.add(ph);
            s_S.add(nd.S);
            s_phit.add(nd.phit);
            s_int.add(kint * phi * (R(1) - phi));                        // Eq. 67 integrand
            ++nodes;
            const bool finite = isfinite(phi) && isfinite(nd.dcA) && isfinite(nd.dcB) && isfinite(ph) &&
                                isfinite(nd.S) && isfinite(umag) && isfinite(nd.phit);
            bad += finite ? 0 : 1;
            if (isfinite(umag)) umax = umag > umax ? umag : umax;
            if constexpr (kTwoD<LAT>) quads += euler_quads4(phi_field, int(x), int(y), P);
            on = phi >= R(0.5);
        }
        if constexpr (!kTwoD<LAT>) {
            if (bits) {
                const unsigned word = __ballot_sync(0xffffffffu, on);
                if (lane == 0) bits[base >> 5] = word;
            }
        }
    }
    double acc[LBM_NRED_DEV];
    acc[0] = s_phi.value();
    acc[1] = s_dcA.value() + double(nodes) * P.c0[0];
    acc[2] = s_dcB.value() + double(nodes) * P.c0[1];
    acc[3] = s_p.value();
    acc[4] = s_S.value();
    acc[5] = double(umax);
    acc[6] = s_phit.value();
    acc[7] = double(bad);
    acc[8] = s_int.value();
    acc[9] = 0.25 * double(quads);
    // block reduction: warp shuffles, then one warp over the warp results
    __shared__ double sm[LBM_NRED_DEV][32];
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
    return dim3((P.nx + bx - 1) / bx, P.ny, P.z_hi - P.z_lo);
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
    template <int LAT>
    static void plane_phi(const DevParams& P, const StateView& st, int mode, int z, void* out, cudaStream_t s) {
        int bx; dim3 grid = node_grid(P, bx);
        grid.z = 1;
        R* o = static_cast<R*>(out);
        LBM_MODE_SWITCH(mode, plane_phi_kernel<T, LAT, M><<<grid, bx, 0, s>>>(P, st, z, o));
    }
    // the per-node step kernel; with flow, the phi pass of the same step must precede it
    template <int LAT, bool FLOW>
    static void step(const DevParams& P, const StateView& st, const StateView& out, int mode, void* phi_work,
                     cudaStream_t s) {
        int bx; const dim3 grid = node_grid(P, bx);
        R* phi = static_cast<R*>(phi_work);
        // MRT in an instance of its own: its 19 x 19 transform would raise every instance's registers
        if constexpr (FLOW) {
            if (P.coll == 2) {
                LBM_MODE_SWITCH(mode, step_kernel<T, LAT, FLOW, M, 2><<<grid, bx, 0, s>>>(P, st, out, phi));
                return;
            }
        }
        LBM_MODE_SWITCH(mode, step_kernel<T, LAT, FLOW, M, -1><<<grid, bx, 0, s>>>(P, st, out, phi));
    }
    static void fused(const DevParams& P, const StateView& src, const StateView& dst, int zchunk, cudaStream_t s) {
        const dim3 block(FX, FY);
        const dim3 grid((P.nx + FX - 1) / FX, (P.ny + FY - 1) / FY, (P.z_hi - P.z_lo + zchunk - 1) / zchunk);
        constexpr size_t smem = fused_smem_bytes<T>();
        // instances per flow collision (see fused_flow_kernel)
        if (P.coll == 2) {
            launch_fused_coll<2>(P, src, dst, zchunk, grid, block, smem, s);
            return;
        }
        if constexpr (is16<T>()) {
            if (P.coll == 1) {
                launch_fused_coll<1>(P, src, dst, zchunk, grid, block, smem, s);
                return;
            }
        }
        launch_fused_coll<0>(P, src, dst, zchunk, grid, block, smem, s);
    }
    template <int COLL>
    static void launch_fused_coll(const DevParams& P, const StateView& src, const StateView& dst, int zchunk,
                                  dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
        // opt in to more than 48 KB of dynamic shared memory, once per device (a repeated
        // call from a racing thread is harmless)
        static unsigned long long configured = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !(configured & (1ull << dev))) {
            cudaFuncSetAttribute(fused_flow_kernel<T, COLL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
            cudaFuncSetAttribute(fused_flow_kernel<T, COLL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
            configured |= 1ull << dev;
        }
        const bool slab = P.z_lo != 0 || P.z_hi != P.nz || P.wall_zlo != P.wall_z || P.wall_zhi != P.wall_z;
        if (slab) fused_flow_kernel<T, COLL, true><<<grid, block, smem, s>>>(P, src, dst, zchunk);
        else fused_flow_kernel<T, COLL, false><<<grid, block, smem, s>>>(P, src, dst, zchunk);
    }
    template <int LAT, bool FLOW>
    static void fields(const DevParams& P, const StateView& st, int mode, void* phi_work, FieldPtrs out,
                       cudaStream_t s) {
        int bx; const dim3 grid = node_grid(P, bx);
        R* phi = static_cast<R*>(phi_work);
        if constexpr (FLOW) { LBM_MODE_SWITCH(mode, phi_kernel<T, LAT, M><<<grid, bx, 0, s>>>(P, st, phi)); }
        LBM_MODE_SWITCH(mode, fields_kernel<T, LAT, FLOW, M><<<grid, bx, 0, s>>>(P, st, phi, out));
    }
    // Blocks of 256 threads of ``kernel`` that the device holds at once, at most ``cap``: a
    // grid-stride kernel launched with more would run its last blocks in a partial wave.
    template <class K>
    static int resident_blocks(K kernel, int cap) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            return cap;
        }
        const long long n = (long long)per_sm * sms;
        return (n > 0 && n < cap) ? int(n) : cap;
    }
    // Fills ``nblocks`` block partials: the grid-stride kernels run with the blocks the device
    // holds at once and the partials of the blocks beyond are zeroed.
    template <int LAT, bool FLOW>
    static void reduce(const DevParams& P, const StateView& st, int mode, void* phi_work, void* bits_work,
                       double* partials, int nblocks, cudaStream_t s) {
        R* phi = static_cast<R*>(phi_work);
        unsigned* bits = static_cast<unsigned*>(bits_work);
        if constexpr (FLOW || kTwoD<LAT>) {
            int bx; const dim3 grid = node_grid(P, bx);
            LBM_MODE_SWITCH(mode, phi_kernel<T, LAT, M><<<grid, bx, 0, s>>>(P, st, phi));
        }
        int nb = nblocks;
        LBM_MODE_SWITCH(mode, {
            nb = resident_blocks(reduce_kernel<T, LAT, FLOW, M>, nblocks);
            reduce_kernel<T, LAT, FLOW, M><<<nb, 256, 0, s>>>(P, st, phi, bits, partials);
        });
        if (nb < nblocks)
            cudaMemsetAsync(partials + (size_t)nb * LBM_NRED_DEV, 0, (size_t)(nblocks - nb) * LBM_NRED_DEV * sizeof(double),
                            s);
        // the 3D Euler count needs the bit field of the whole lattice (not kept for a slab)
        if constexpr (!kTwoD<LAT>) {
            if (bits) euler3d_kernel<T><<<resident_blocks(euler3d_kernel<T>, nblocks), 256, 0, s>>>(P, bits, partials);
        }
    }
};

// Dispatch over (lattice, flow) for one storage type.
#define LBM_DEFINE_LAUNCHERS(T, SUFFIX)                                                                   \
    void launch_init_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, bool pull,      \
                              const double* a, const double* b, const double* c, cudaStream_t s) {        \
        if (lat == LAT_D2Q5) Launchers<T>::init<LAT_D2Q5, false>(P, st, pull, a, b, c, s);                 \
        else if (lat == LAT_D2Q9) Launchers<T>::init<LAT_D2Q9, false>(P, st, pull, a, b, c, s);            \
        else if (lat == LAT_D3Q19 && flow) Launchers<T>::init<LAT_D3Q19, true>(P, st, pull, a, b, c, s);   \
        else if (lat == LAT_D3Q19) Launchers<T>::init<LAT_D3Q19, false>(P, st, pull, a, b, c, s);          \
        else if (flow) Launchers<T>::init<LAT_D3Q7, true>(P, st, pull, a, b, c, s);                        \
        else Launchers<T>::init<LAT_D3Q7, false>(P, st, pull, a, b, c, s);                                 \
    }                                                                                                     \
    void launch_phi_##SUFFIX(const DevParams& P, const StateView& st, int lat, int mode, void* phi,       \
                             cudaStream_t s) {                                                            \
        if (lat == LAT_D2Q5) Launchers<T>::phi<LAT_D2Q5>(P, st, mode, phi, s);                             \
        else if (lat == LAT_D2Q9) Launchers<T>::phi<LAT_D2Q9>(P, st, mode, phi, s);                        \
        else if (lat == LAT_D3Q19) Launchers<T>::phi<LAT_D3Q19>(P, st, mode, phi, s);                      \
        else Launchers<T>::phi<LAT_D3Q7>(P, st, mode, phi, s);                                             \
    }                                                                                                     \
    void launch_plane_phi_##SUFFIX(const DevParams& P, const StateView& st, int lat, int mode, int z,    \
                                   void* out, cudaStream_t s) {                                           \
        if (lat == LAT_D2Q5) Launchers<T>::plane_phi<LAT_D2Q5>(P, st, mode, z, out, s);                    \
        else if (lat == LAT_D2Q9) Launchers<T>::plane_phi<LAT_D2Q9>(P, st, mode, z, out, s);               \
        else if (lat == LAT_D3Q19) Launchers<T>::plane_phi<LAT_D3Q19>(P, st, mode, z, out, s);             \
        else Launchers<T>::plane_phi<LAT_D3Q7>(P, st, mode, z, out, s);                                    \
    }                                                                                                     \
    void launch_step_##SUFFIX(const DevParams& P, const StateView& st, const StateView& out, int lat,     \
                              bool flow, int mode, void* phi, cudaStream_t s) {                            \
        if (lat == LAT_D2Q5) Launchers<T>::step<LAT_D2Q5, false>(P, st, out, mode, phi, s);                \
        else if (lat == LAT_D2Q9) Launchers<T>::step<LAT_D2Q9, false>(P, st, out, mode, phi, s);           \
        else if (lat == LAT_D3Q19 && flow) Launchers<T>::step<LAT_D3Q19, true>(P, st, out, mode, phi, s);  \
        else if (lat == LAT_D3Q19) Launchers<T>::step<LAT_D3Q19, false>(P, st, out, mode, phi, s);         \
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
        else if (lat == LAT_D2Q9) Launchers<T>::fields<LAT_D2Q9, false>(P, st, mode, phi, out, s);         \
        else if (lat == LAT_D3Q19 && flow) Launchers<T>::fields<LAT_D3Q19, true>(P, st, mode, phi, out, s); \
        else if (lat == LAT_D3Q19) Launchers<T>::fields<LAT_D3Q19, false>(P, st, mode, phi, out, s);       \
        else if (flow) Launchers<T>::fields<LAT_D3Q7, true>(P, st, mode, phi, out, s);                     \
        else Launchers<T>::fields<LAT_D3Q7, false>(P, st, mode, phi, out, s);                              \
    }                                                                                                     \
    void launch_reduce_##SUFFIX(const DevParams& P, const StateView& st, int lat, bool flow, int mode,    \
                                void* phi, void* bits, double* partials, int nblocks, cudaStream_t s) {   \
        if (lat == LAT_D2Q5) Launchers<T>::reduce<LAT_D2Q5, false>(P, st, mode, phi, bits, partials, nblocks, s); \
        else if (lat == LAT_D2Q9)                                                                         \
            Launchers<T>::reduce<LAT_D2Q9, false>(P, st, mode, phi, bits, partials, nblocks, s);           \
        else if (lat == LAT_D3Q19 && flow)                                                                \
            Launchers<T>::reduce<LAT_D3Q19, true>(P, st, mode, phi, bits, partials, nblocks, s);           \
        else if (lat == LAT_D3Q19)                                                                        \
            Launchers<T>::reduce<LAT_D3Q19, false>(P, st, mode, phi, bits, partials, nblocks, s);          \
        else if (flow) Launchers<T>::reduce<LAT_D3Q7, true>(P, st, mode, phi, bits, partials, nblocks, s); \
        else Launchers<T>::reduce<LAT_D3Q7, false>(P, st, mode, phi, bits, partials, nblocks, s);          \
    }

}  // namespace lbm
