// Device-side building blocks of the coupled step: lattice tables, storage codecs,
// AA-pattern addressing and the per-node physics of §3. Included by the per-storage
// translation units; nothing here launches work.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {

// ------------------------------------------------------------------------------------
// Parameters as the kernels see them (derived once on the host from lbm_params).
// Model coefficients in the working precision of a kernel (filled on the host from the
// FP64 values below), so that FP32 kernels never convert an FP64 parameter per node.
template <class R>
struct Coef {
    R lam, kphi, c0[2], dc[2], om_g, M0[2], M1[2], om_f, om_fm, sw15, inv_W2, g[3];
    R mrt[19];            // MRT: rate / |row|^2 of each moment of the D3Q19 basis
};

struct DevParams {
    int nx, ny, nz;
    int wall_x, wall_z, source_off;
    int coll;             // flow collision: 0 BGK (Eq. 36), 1 TRT, 2 MRT
    long long n;          // nodes
    long long plane;      // elements between two population planes (n rounded up)
    double W, lam;
    double kphi;          // M_phi / W^2 = 1 / tau_phi (§2.2)
    double c0[2], c1[2];  // c_0^eq, c_1^eq per component
    double dc[2];         // c_1^eq - c_0^eq
    double om_g;          // 1 / (M_phi / c_s^2 + 1/2)  (Eq. 46 with M_phi = tau_g c_s^2)
    double M0[2], M1[2];  // mobilities of phase 0 and 1 per component (§2.3)
    double inv_cs2;       // 1 / c_s^2 of the scalar lattice
    double om_f;          // 1 / (nu / c_s^2 + 1/2)  (Eq. 36), c_s^2 = 1/3
    double om_fm;         // TRT rate of the odd part: 1 / (Lambda / (1/om_f - 1/2) + 1/2)
    double mrt[19];       // MRT rate of each moment divided by the squared norm of its row
    double sw15;          // (3/2) sigma W  (Eq. 34)
    double inv_W2;
    double g[3];          // buoyancy per unit phi
    double f_scale, inv_f_scale;
    Coef<float> cf;
    Coef<double> cd;
};

template <class R> __host__ __device__ __forceinline__ const Coef<R>& coef(const DevParams& P);
template <> __host__ __device__ __forceinline__ const Coef<float>& coef<float>(const DevParams& P) { return P.cf; }
template <> __host__ __device__ __forceinline__ const Coef<double>& coef<double>(const DevParams& P) { return P.cd; }

// Pointers of one state buffer: population planes in the storage type, plus the FP32
// rest-population planes used by 16-bit storage. ``plane`` lists every population plane
// (f_0..f_18, then the Q planes of g, h^A and h^B: Planes<LAT>) so that a kernel can
// address population k of node n as plane[k] + n, the pointer coming straight from the
// kernel's parameter space.
constexpr int kPlanes = 19 + 3 * 19;   // room for D3Q19 scalar sets
struct StateView {
    void* f;      // 19 planes (flow only)
    void* g;      // Q planes
    void* hA;
    void* hB;
    float* rest;  // 4 FP32 planes (g_0, hA_0, hB_0, f_0) for 16-bit storage, else nullptr
    void* plane[kPlanes];
};

enum { LAT_D2Q5 = 0, LAT_D3Q7 = 1, LAT_D3Q19 = 2, LAT_D2Q9 = 3 };

// ------------------------------------------------------------------------------------
// Velocity sets. Scalar sets: k = 0 at rest, then +x, -x, +y, -y (, +z, -z).
// Flow set: D3Q19 in the order of the paper's table (§3). For every set the opposite of
// k > 0 is k + 1 for odd k and k - 1 for even k.
template <int LAT> struct Scalar;

template <> struct Scalar<LAT_D2Q5> {
    static constexpr int Q = 5;
    __host__ __device__ static constexpr int ex(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int k) { return k == 3 ? 1 : (k == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

template <> struct Scalar<LAT_D3Q7> {
    static constexpr int Q = 7;
    __host__ __device__ static constexpr int ex(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int k) { return k == 3 ? 1 : (k == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int k) { return k == 5 ? 1 : (k == 6 ? -1 : 0); }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 0.25 : 0.125; }
    __host__ __device__ static constexpr double cs2() { return 0.25; }
};

struct D3Q19 {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int ex(int k) {
        return (k == 1 || k == 7 || k == 9 || k == 13 || k == 15) ? 1
             : (k == 2 || k == 8 || k == 10 || k == 14 || k == 16) ? -1 : 0;
    }
    __host__ __device__ static constexpr int ey(int k) {
        return (k == 3 || k == 7 || k == 11 || k == 14 || k == 17) ? 1
             : (k == 4 || k == 8 || k == 12 || k == 13 || k == 18) ? -1 : 0;
    }
    __host__ __device__ static constexpr int ez(int k) {
        return (k == 5 || k == 9 || k == 11 || k == 16 || k == 18) ? 1
             : (k == 6 || k == 10 || k == 12 || k == 15 || k == 17) ? -1 : 0;
    }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

// d'Humieres' orthogonal moment basis of D3Q19, evaluated on the velocities above: row i
// is density, energy, energy square, (momentum, energy flux) per axis, (3 p_xx, pi_xx),
// (p_ww, pi_ww), p_xy, p_yz, p_xz, m_x, m_y, m_z. Rows are orthogonal; norm(i) = |row i|^2.
struct MRT19 {
    __host__ __device__ static constexpr double m(int i, int k) {
        const double cx = D3Q19::ex(k), cy = D3Q19::ey(k), cz = D3Q19::ez(k);
        const double c2 = cx * cx + cy * cy + cz * cz;
        switch (i) {
            case 0: return 1.0;
            case 1: return 19.0 * c2 - 30.0;
            case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
            case 3: return cx;
            case 4: return (5.0 * c2 - 9.0) * cx;
            case 5: return cy;
            case 6: return (5.0 * c2 - 9.0) * cy;
            case 7: return cz;
            case 8: return (5.0 * c2 - 9.0) * cz;
            case 9: return 3.0 * cx * cx - c2;
            case 10: return (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2);
            case 11: return cy * cy - cz * cz;
            case 12: return (3.0 * c2 - 5.0) * (cy * cy - cz * cz);
            case 13: return cx * cy;
            case 14: return cy * cz;
            case 15: return cx * cz;
            case 16: return (cy * cy - cz * cz) * cx;
            case 17: return (cz * cz - cx * cx) * cy;
            default: return (cx * cx - cy * cy) * cz;
        }
    }
    __host__ __device__ static constexpr double norm(int i) {
        double s = 0.0;
        for (int k = 0; k < 19; ++k) s += m(i, k) * m(i, k);
        return s;
    }
};

// D3Q19 as the lattice of phi, c^A, c^B: the paper's choice for every equation (§3).
template <> struct Scalar<LAT_D3Q19> {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int ex(int k) { return D3Q19::ex(k); }
    __host__ __device__ static constexpr int ey(int k) { return D3Q19::ey(k); }
    __host__ __device__ static constexpr int ez(int k) { return D3Q19::ez(k); }
    __host__ __device__ static constexpr double w(int k) { return D3Q19::w(k); }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

// D2Q9 as the lattice of phi, c^A, c^B in 2D (the paper's choice in 2D, §3): rest, the four
// axis directions, then the diagonals, opposite pairs adjacent as in every set here.
template <> struct Scalar<LAT_D2Q9> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int ex(int k) {
        return (k == 1 || k == 5 || k == 7) ? 1 : ((k == 2 || k == 6 || k == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int k) {
        return (k == 3 || k == 5 || k == 8) ? 1 : ((k == 4 || k == 6 || k == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

// First plane of g, h^A, h^B in StateView::plane for a scalar lattice.
template <int LAT> struct Planes {
    static constexpr int G = 19, HA = 19 + Scalar<LAT>::Q, HB = 19 + 2 * Scalar<LAT>::Q;
};

// ------------------------------------------------------------------------------------
// Storage codecs. Real is the arithmetic type (double for FP64 storage, float otherwise).
template <class T> struct RealOf { using type = float; };
template <> struct RealOf<double> { using type = double; };

// Which population set a plane belongs to, for the 16-bit deviation encoding.
enum { SET_F = 0, SET_G = 1, SET_H = 2 };
constexpr float kHScale = 64.0f;       // 16-bit h_k / w_k scale (h_k ~ w_k mu, mu ~ 1e-3..1e-2)
constexpr float kFScale = 1024.0f;     // 16-bit f_k / w_k scale (f_k ~ w_k (p_h + 3 e.u) ~ 1e-3 w_k)

template <class T> struct Codec {
    // plain FP32 / FP64 storage
    template <int SET>
    __device__ static typename RealOf<T>::type load(const T* p, double, const DevParams&) { return *p; }
    template <int SET>
    __device__ static void store(T* p, typename RealOf<T>::type v, double, const DevParams&) { *p = v; }
};

__device__ inline float to_f(__half v) { return __half2float(v); }
__device__ inline float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class T> __device__ inline T from_f(float v);
template <> __device__ inline __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ inline __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// 16-bit storage holds each moving population P_k as its scaled deviation q_k:
//   f: P = (w / kFScale) q,  g: P = w (q + 1/2),  h: P = (w / kHScale) q,
// so that q is O(1) for every set. Kernels load q as it is (a Node of a 16-bit state holds
// q_k for k > 0 and the FP32 rest population for k = 0), run the collision on q (the
// BGK update is affine, so it keeps its form with the weights divided out) and store q.
template <class H> struct Codec16 {
    // population = scale * q + offset
    template <int SET> __host__ __device__ static constexpr double scale(double w) {
        return SET == SET_F ? w / kFScale : (SET == SET_G ? w : w / kHScale);
    }
    template <int SET> __host__ __device__ static constexpr double offset(double w) {
        return SET == SET_G ? 0.5 * w : 0.0;
    }
    template <int SET>
    __device__ static float load(const H* p, double, const DevParams&) { return to_f(*p); }
    // encode a population given in natural units (initial state)
    template <int SET>
    __device__ static void store(H* p, float v, double w, const DevParams&) {
        float q;
        if (SET == SET_F) q = v * float(kFScale / w);
        else if (SET == SET_G) q = v * float(1.0 / w) - 0.5f;
        else q = v * float(kHScale / w);
        *p = from_f<H>(q);
    }
    // Store q and return the stored value read back, round16(q): the caller subtracts the
    // moving populations as stored from the node's conserved total to set its FP32 rest
    // population, so 16-bit rounding never changes the node's sums.
    __device__ static float store_q_back(H* p, float q) {
        const H h = from_f<H>(q);
        *p = h;
        return to_f(h);
    }
};
template <> struct Codec<__half> : Codec16<__half> {};
template <> struct Codec<__nv_bfloat16> : Codec16<__nv_bfloat16> {};

template <class T> constexpr bool is16() { return sizeof(T) == 2; }

// ------------------------------------------------------------------------------------
// Pointwise model of §2 (Real precision).
template <class R> __device__ __forceinline__ R interp_p(R f) { return f * f * (R(3) - R(2) * f); }
template <class R> __device__ __forceinline__ R interp_dp(R f) { return R(6) * f * (R(1) - f); }
template <class R> __device__ __forceinline__ R dwell_d(R f) { return R(16) * f * (R(1) - f) * (R(1) - R(2) * f); }

// Eq. 33 written as mu = (c - c_0^eq) - p(phi) (c_1^eq - c_0^eq), since p(1 - phi) = 1 - p(phi).
// The kernels carry the composition as its deviation dc = c - c_0^eq (see the h_0 storage).
template <class R> __device__ __forceinline__ R closure_dev(R dc, R p, int a, const DevParams& P) {
    return dc - p * coef<R>(P).dc[a];
}
// Eq. 35 with Delta omega of Eq. 20 = sum mu (c_1^eq - c_0^eq)
template <class R> __device__ __forceinline__ R source(R phi, R muA, R muB, const DevParams& P) {
    if (P.source_off) return R(0);
    R dom = muA * coef<R>(P).dc[0] + muB * coef<R>(P).dc[1];
    return coef<R>(P).kphi * (-dwell_d(phi) + coef<R>(P).lam * interp_dp(phi) * dom);
}

// ------------------------------------------------------------------------------------
// Addressing. Node index of (x, y, z) with x fastest.
// Node indices are 32-bit (the host rejects lattices of 2^31 nodes or more); offsets into
// the population planes are formed in 64 bits.
__device__ __forceinline__ int node_of(int x, int y, int z, const DevParams& P) {
    return (z * P.ny + y) * P.nx + x;
}
// Population slot of a node: element node of population plane slot.
struct Slot { int node; int slot; };

// Element of population slot s.slot (k or opp(k): the slot is one of these two constants) of
// the set whose first plane is B, at node s.node.
template <class T, int B>
__device__ __forceinline__ T* element(const StateView& st, int k, Slot s) {
    T* base = static_cast<T*>(s.slot == k ? st.plane[B + k] : st.plane[B + opp(k)]);
    return base + s.node;
}

// Load / store one population of a scalar set (first plane B); with 16-bit storage the rest
// population lives in FP32 rest plane RP (g: 0, h^A: 1, h^B: 2, f: 3).
template <class T, int SET, int LAT, int B, int RP>
__device__ __forceinline__ typename RealOf<T>::type load_scalar(const StateView& st, int k, Slot s,
                                                                const DevParams& P) {
    if (is16<T>() && k == 0) return st.rest[RP * P.plane + s.node];
    return Codec<T>::template load<SET>(element<T, B>(st, k, s), Scalar<LAT>::w(k), P);
}
template <class T, int SET, int LAT, int B, int RP>
__device__ __forceinline__ void store_scalar(const StateView& st, int k, Slot s, typename RealOf<T>::type v,
                                             const DevParams& P) {
    if (is16<T>() && k == 0) { st.rest[RP * P.plane + s.node] = float(v); return; }
    Codec<T>::template store<SET>(element<T, B>(st, k, s), v, Scalar<LAT>::w(k), P);
}


}  // namespace lbm
