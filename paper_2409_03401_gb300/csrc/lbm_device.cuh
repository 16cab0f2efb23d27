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
    int wall_zlo, wall_zhi;   // z walls at each end (a slab has them only where the lattice ends)
    int z_lo, z_hi;           // planes the kernels advance, [z_lo, z_hi): (0, nz), or a slab's own
    const void* phi_ghost[2]; // slab: phi (Real, nx * ny) of the planes z_lo - 1 and z_hi, which
                              // belong to the neighbouring slabs; nullptr where a wall bounds z
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
    float* rest;  // 5 FP32 planes (g_0, hA_0, hB_0, f_0, f_0 of odd time levels in place) for
                  // 16-bit storage, else nullptr
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

// Which population set a plane belongs to, for the 16-bit encodings.
enum { SET_F = 0, SET_G = 1, SET_H = 2 };

template <class T> struct Codec {
    // plain FP32 / FP64 storage
    template <int SET>
    __device__ static typename RealOf<T>::type load(const T* p, double, const DevParams&) { return *p; }
    template <int SET>
    __device__ static void store(T* p, typename RealOf<T>::type v, double, const DevParams&) { *p = v; }
};

// 16-bit population storage. Every moving population P_k (k > 0) is held as its value per
// unit weight, x_k = P_k / w_k - o, with o = 1/2 for g (phi lies in [0, 1]) and o = 0 for h,
// and for f as the deviation from its writer's rest population, x_k = f_k / w_k - f_0 / w_0
// (f_0 ~ w_0 p_h, so x_k ~ e_k . u: the pressure, which can exceed u by an order of
// magnitude, is not rounded). Kernels decode x_k to FP32, collide on it (every equilibrium
// and source term carries w_k, so the update keeps its affine form per unit weight) and
// encode the result. The rest populations stay FP32.
//
// Store16 (storage LBM_F16) chooses a format per set from the range each set spans:
//   g: 16-bit fixed point, x = (n - 32768) / 2^15 for the stored n in [0, 65535], i.e.
//      x in [-1, 1) with a uniform step of 3.05e-5 (IEEE FP16's step near |x| = 1/2, where
//      the bulk phases sit, is 8 times coarser; phi's rounding noise drives the capillary
//      force, so it sets the velocity error); values beyond saturate, which a stable run
//      (|u| well below 0.1, phi within [0, 1] up to small overshoots) never reaches;
//   f: IEEE FP16 of 1024 x (x ~ e.u after the reference is taken off);
//   h: IEEE FP16 of 64 x (x ~ mu + c e.u / c_s^2).
// An unstable run still shows: its FP32 rest populations go non-finite.
// __nv_bfloat16 (storage LBM_BF16) stores every x as BF16 (8-bit significand).
struct Store16 { unsigned short bits; };

namespace fmt16 {
// 16-bit fixed point over [-1, 1): 1.5 * 2^23 + n is exact in FP32, so one FMA decodes
constexpr float kMagic = 12582912.0f;                             // 1.5 * 2^23
__device__ __forceinline__ float q15_dec(unsigned w) {
    return fmaf(__uint_as_float(0x4B400000u | (w & 0xFFFFu)), 3.0517578125e-05f, -385.0f);
}
__device__ __forceinline__ unsigned short q15_enc(float v) {
    float y = fmaf(v, 32768.0f, kMagic + 32768.0f);               // rounds to the nearest integer
    y = fminf(fmaxf(y, kMagic), kMagic + 65535.0f);
    return (unsigned short)(__float_as_uint(y) & 0xFFFFu);
}
}  // namespace fmt16

constexpr float kF16FScale = 1024.0f;  // Store16 f: IEEE FP16 of 1024 x
constexpr float kF16HScale = 64.0f;  // Store16 h: IEEE FP16 of 64 x (x ~ mu stays clear of subnormals)

// Each set is stored in units of r = unit * x (unit: f 1024, g 1, h 64 for Store16; 1 for
// BF16); dec returns r, enc takes r.
template <class H> struct Codec16;
template <> struct Codec16<Store16> {
    template <int SET> __host__ __device__ static constexpr float unit() {
        return SET == SET_F ? kF16FScale : (SET == SET_H ? kF16HScale : 1.0f);
    }
    template <int SET> __device__ static float dec(Store16 v) {
        if (SET == SET_G) return fmt16::q15_dec(v.bits);
        return __half2float(__ushort_as_half(v.bits));
    }
    template <int SET> __device__ static Store16 enc(float r) {
        if (SET == SET_G) return Store16{fmt16::q15_enc(r)};
        return Store16{__half_as_ushort(__float2half_rn(r))};
    }
};
template <> struct Codec16<__nv_bfloat16> {
    template <int SET> __host__ __device__ static constexpr float unit() { return 1.0f; }
    template <int SET> __device__ static float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
    template <int SET> __device__ static __nv_bfloat16 enc(float r) { return __float2bfloat16_rn(r); }
};

// The codec behind the node loaders: population = scale * r + offset, r as stored.
template <class H> struct Codec16Pop : Codec16<H> {
    template <int SET> __host__ __device__ static constexpr double scale(double w) {
        return w / Codec16<H>::template unit<SET>();
    }
    template <int SET> __host__ __device__ static constexpr double offset(double w) {
        return SET == SET_G ? 0.5 * w : 0.0;
    }
    template <int SET>
    __device__ static float load(const H* p, double, const DevParams&) { return Codec16<H>::template dec<SET>(*p); }
    // encode a population given in natural units (initial state; f with a zero reference)
    template <int SET>
    __device__ static void store(H* p, float v, double w, const DevParams&) {
        constexpr float u = Codec16<H>::template unit<SET>();
        const float r = SET == SET_G ? v * float(u / w) - 0.5f * u : v * float(u / w);
        *p = Codec16<H>::template enc<SET>(r);
    }
    // Store r and return the value as stored, dec(enc(r)): the caller subtracts the moving
    // populations as stored from the node's conserved total to set the FP32 rest population
    // of g and h, so 16-bit rounding never changes those sums.
    template <int SET>
    __device__ static float store_back(H* p, float r) {
        const H h = Codec16<H>::template enc<SET>(r);
        *p = h;
        return Codec16<H>::template dec<SET>(h);
    }
};
template <> struct Codec<Store16> : Codec16Pop<Store16> {};
template <> struct Codec<__nv_bfloat16> : Codec16Pop<__nv_bfloat16> {};

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
