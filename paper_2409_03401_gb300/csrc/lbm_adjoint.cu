// Discrete adjoint of the coupled step without flow (reverse mode, written by hand).
//
// Forward step t (per node x): incoming populations P_t(x, .) -> local BGK collision C
// (Eqs. 20, 33, 35, 46-51) -> P*_t(x, .) -> streaming: P_{t+1}(x + e_k, k) = P*_t(x, k),
// or P_{t+1}(x, opp(k)) = P*_t(x, k) across a wall. With Lambda_t = dL/dP_t:
//   dL/dP*_t(x, k) = Lambda_{t+1} at the node and slot P*_t(x, k) streams to,
//   Lambda_t(x, .) = J_C(P_t(x))^T dL/dP*_t(x, .),
//   dL/dtheta     += sum_x (dC/dtheta)^T dL/dP*_t(x, .).
// Lambda is kept in canonical layout: plane (set * Q + k), set = g, h^A, h^B, element x.
// The forward states are read in the AA layout of their time level.
#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kAdjBlocks = 1216;   // grid-stride blocks; one row of partials per block
constexpr int kNTheta = 5;         // dL/dM[0][A], dL/dM[0][B], dL/dM[1][A], dL/dM[1][B], dL/dM_phi

template <class R> __device__ __forceinline__ R dwell_dd(R f) { return R(16) * (R(1) - R(6) * f + R(6) * f * f); }
template <class R> __device__ __forceinline__ R interp_ddp(R f) { return R(6) * (R(1) - R(2) * f); }

// (x, y, z) of linear node id
__device__ __forceinline__ void coords(long long id, const DevParams& P, int& x, int& y, int& z) {
    x = int(id % P.nx);
    y = int((id / P.nx) % P.ny);
    z = int(id / ((long long)P.nx * P.ny));
}

// Reverse of S = K B(phi~, mu~), B = -omega_dw'(phi~) + lambda p'(phi~) Delta omega(mu~),
// mu~_a = dc_a - p(phi~) Delta c_a: adds to phitb, dcb[2] and to the M_phi gradient.
// The M_phi derivative of S is B / W^2; ``SbB`` receives S-bar * B (the 1/W^2 is applied
// once per block).
template <class R>
__device__ __forceinline__ void source_adjoint(R phit, R dcA, R dcB, R Sb, const DevParams& P,
                                               R& phitb, R& dcAb, R& dcBb, R& SbB) {
    if (P.source_off) return;
    const R pt = interp_p(phit), dpt = interp_dp(phit);
    const R muA = closure_dev(dcA, pt, 0, P), muB = closure_dev(dcB, pt, 1, P);
    const R dom = muA * coef<R>(P).dc[0] + muB * coef<R>(P).dc[1];
    const R B = -dwell_d(phit) + coef<R>(P).lam * dpt * dom;
    SbB += Sb * B;                                              // K = M_phi / W^2
    const R Bb = Sb * coef<R>(P).kphi;
    phitb += Bb * (-dwell_dd(phit) + coef<R>(P).lam * interp_ddp(phit) * dom);
    const R domb = Bb * coef<R>(P).lam * dpt;
    const R muAb = domb * coef<R>(P).dc[0], muBb = domb * coef<R>(P).dc[1];
    dcAb += muAb;
    dcBb += muBb;
    phitb += -dpt * (coef<R>(P).dc[0] * muAb + coef<R>(P).dc[1] * muBb);
}

// Per-node parameter-gradient terms, summed per block in FP64 and scaled there:
//   acc[0..1] = M-bar_a (1 - phi), acc[2..3] = M-bar_a phi   (dL/dM[0][a], dL/dM[1][a])
//   acc[4]    = S-bar B           (x 1/W^2 -> part of dL/dM_phi through the source)
//   acc[5]    = om_g-bar          (x d om_g / d M_phi = -om_g^2 / c_s^2)
constexpr int kNAcc = 6;

// Transpose of the local collision Jacobian at the incoming state nd, applied to the
// adjoint of the post-collision values (ag, ahA, ahB); writes the adjoint of the incoming
// values (gb, hAb, hBb) and adds the node's parameter-gradient terms to acc[kNAcc].
template <class T, int LAT>
__device__ __forceinline__ void collide_adjoint(const Node<T, LAT, false>& nd,
                                                const typename RealOf<T>::type* ag,
                                                const typename RealOf<T>::type* ahA,
                                                const typename RealOf<T>::type* ahB,
                                                typename RealOf<T>::type* gb, typename RealOf<T>::type* hAb,
                                                typename RealOf<T>::type* hBb, typename RealOf<T>::type* acc,
                                                const DevParams& P) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    constexpr int Q = L::Q;
    const R inv_cs2 = R(1.0 / L::cs2());
    // forward quantities (as in collide_store with u = 0)
    const R S = nd.S;
    const R phi = nd.phi();
    const R p = interp_p(phi), dp = interp_dp(phi);
    const R mu[2] = {closure_dev(nd.dcA, p, 0, P), closure_dev(nd.dcB, p, 1, P)};
    const R dcv[2] = {nd.dcA, nd.dcB};
    const R omg = coef<R>(P).om_g;
    const R* h[2] = {nd.hA, nd.hB};
    const R* ah[2] = {ahA, ahB};
    R* hb[2] = {hAb, hBb};

    // g* = (1 - om_g) g + om_g w phi + w S (1 - om_g / 2)
    R Gw = R(0), omgb = R(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const R w = R(L::w(k));
        gb[k] = (R(1) - omg) * ag[k];
        Gw += w * ag[k];
        omgb += ag[k] * (w * phi - R(0.5) * w * S - nd.g[k]);
    }
    R phib = omg * Gw;
    R Sb = Gw * (R(1) - R(0.5) * omg);
    acc[5] += omgb;
    R dcb[2] = {R(0), R(0)};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const R M = coef<R>(P).M0[a] * (R(1) - phi) + coef<R>(P).M1[a] * phi;
        const R om = recip(M * inv_cs2 + R(0.5));
        R omb = R(0), mub = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R w = R(L::w(k));
            const R heq = k == 0 ? dcv[a] - (R(1) - w) * mu[a] : w * mu[a];
            hb[a][k] = (R(1) - om) * ah[a][k];
            omb += ah[a][k] * (heq - h[a][k]);
            if (k == 0) { dcb[a] += om * ah[a][0]; mub += -om * (R(1) - w) * ah[a][0]; }
            else mub += om * w * ah[a][k];
        }
        const R Mb = omb * (-om * om * inv_cs2);
        acc[a] += Mb * (R(1) - phi);                               // dL/dM[0][a]
        acc[2 + a] += Mb * phi;                                    // dL/dM[1][a]
        phib += Mb * (coef<R>(P).M1[a] - coef<R>(P).M0[a]);
        dcb[a] += mub;                                             // mu = dc - p(phi) Delta c
        phib += -dp * coef<R>(P).dc[a] * mub;
    }
    // phi = phi~ + S / 2
    R phitb = phib;
    Sb += R(0.5) * phib;
    source_adjoint(nd.phit, nd.dcA, nd.dcB, Sb, P, phitb, dcb[0], dcb[1], acc[4]);
    // phi~ = sum g, dc = sum h
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        gb[k] += phitb;
        hAb[k] += dcb[0];
        hBb[k] += dcb[1];
    }
}

// Block sum of the per-node terms in the working precision (a block holds at most a few
// hundred nodes), mapped to the five gradient components and added in FP64 to this
// block's row of partials; rows are summed over steps and blocks by theta_final. One
// thread per block touches FP64, whose throughput is low on this part.
template <class R>
__device__ __forceinline__ void block_accumulate(const R* acc, double* __restrict__ partials, long long row,
                                                 const DevParams& P, double om_g_deriv) {
    __shared__ R sm[kNAcc][32];
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int i = 0; i < kNAcc; ++i) {
        R v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[i][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
        R s[kNAcc];
#pragma unroll
        for (int i = 0; i < kNAcc; ++i) {
            R v = lane < nw ? sm[i][lane] : R(0);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            s[i] = v;
        }
        if (lane == 0) {
            double* pr = partials + row * kNTheta;
            pr[0] += double(s[0]);
            pr[1] += double(s[1]);
            pr[2] += double(s[2]);
            pr[3] += double(s[3]);
            pr[4] += double(s[4]) * P.inv_W2 + double(s[5]) * om_g_deriv;
        }
    }
}

// One reverse step: Lambda_t from Lambda_{t+1} at the state of time t (AA layout, MODE).
// Grid as the forward step: x along threads, y and z along blocks; one node per thread.
template <class T, int LAT, int MODE>
__global__ void __launch_bounds__(kBlockX)
adjoint_step_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ lam_next,
                    typename RealOf<T>::type* __restrict__ lam, double* __restrict__ partials, double om_g_deriv) {
    using R = typename RealOf<T>::type;
    using L = Scalar<LAT>;
    constexpr int Q = L::Q;
    R acc[kNAcc] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x < P.nx) {
        const int self = node_of(x, y, z, P);
        Addr<MODE> ad;
        ad.nb.init(x, y, z, P);
        ad.self = self;
        Node<T, LAT, false> nd;
        nd.gather(st, ad, P);
        nd.moments(P);
        // where the forward step streams P*_t(x, k): the AA odd-step scatter pattern,
        // which sends it to slot k of x + e_k, or to slot opp(k) of x across a wall
        Addr<AA_ODD> fwd;
        fwd.nb = ad.nb;
        fwd.self = self;
        R ag[Q], ahA[Q], ahB[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const Slot s = fwd.dst(k, L::ex(k), L::ey(k), L::ez(k));
            ag[k] = lam_next[(long long)(0 * Q + s.slot) * P.plane + s.node];
            ahA[k] = lam_next[(long long)(1 * Q + s.slot) * P.plane + s.node];
            ahB[k] = lam_next[(long long)(2 * Q + s.slot) * P.plane + s.node];
        }
        R gb[Q], hAb[Q], hBb[Q];
        collide_adjoint<T, LAT>(nd, ag, ahA, ahB, gb, hAb, hBb, acc, P);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            lam[(long long)(0 * Q + k) * P.plane + self] = gb[k];
            lam[(long long)(1 * Q + k) * P.plane + self] = hAb[k];
            lam[(long long)(2 * Q + k) * P.plane + self] = hBb[k];
        }
    }
    const long long row = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_accumulate(acc, partials, row, P, om_g_deriv);
}

// Lambda_T from the adjoint of the output fields phi, mu^A, mu^B at time T.
template <class T, int LAT, int MODE>
__global__ void __launch_bounds__(256)
adjoint_seed_kernel(const DevParams P, const StateView st, const typename RealOf<T>::type* __restrict__ phib_f,
                    const typename RealOf<T>::type* __restrict__ muAb_f,
                    const typename RealOf<T>::type* __restrict__ muBb_f, typename RealOf<T>::type* __restrict__ lam,
                    double* __restrict__ partials) {
    using R = typename RealOf<T>::type;
    constexpr int Q = Scalar<LAT>::Q;
    R acc[kNAcc] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < P.n; id += stride) {
        int x, y, z;
        coords(id, P, x, y, z);
        const int self = int(id);
        Addr<MODE> ad;
        ad.nb.init(x, y, z, P);
        ad.self = self;
        Node<T, LAT, false> nd;
        nd.gather(st, ad, P);
        nd.moments(P);
        const R phi = nd.phi();
        const R dp = interp_dp(phi);
        const R muAb = muAb_f ? muAb_f[self] : R(0), muBb = muBb_f ? muBb_f[self] : R(0);
        R dcAb = muAb, dcBb = muBb;                                 // mu = dc - p(phi) Delta c
        const R phib = (phib_f ? phib_f[self] : R(0)) - dp * (coef<R>(P).dc[0] * muAb + coef<R>(P).dc[1] * muBb);
        R phitb = phib;                                             // phi = phi~ + S / 2
        source_adjoint(nd.phit, nd.dcA, nd.dcB, R(0.5) * phib, P, phitb, dcAb, dcBb, acc[4]);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            lam[(long long)(0 * Q + k) * P.plane + self] = phitb;
            lam[(long long)(1 * Q + k) * P.plane + self] = dcAb;
            lam[(long long)(2 * Q + k) * P.plane + self] = dcBb;
        }
    }
    block_accumulate(acc, partials, blockIdx.x, P, 0.0);
}

// dL/dphi_0 through the initial populations g = w phi0 - w S0/2, h = h^eq(c0, mu0(phi0));
// the piecewise initial compositions (Eq. 66) have zero derivative in phi0.
template <class T, int LAT>
__global__ void __launch_bounds__(256)
adjoint_init_kernel(const DevParams P, const double* __restrict__ phi0, const double* __restrict__ cA0,
                    const double* __restrict__ cB0, const typename RealOf<T>::type* __restrict__ lam,
                    double* __restrict__ phi0b, double* __restrict__ partials) {
    using L = Scalar<LAT>;
    constexpr int Q = L::Q;
    double acc[kNAcc] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < P.n; id += stride) {
        const double ph = phi0[id];
        const double d[2] = {cA0[id] - P.c0[0], cB0[id] - P.c0[1]};
        double Gw = 0.0, mub[2] = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const double w = L::w(k);
            Gw += w * double(lam[(long long)k * P.plane + id]);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const double lh = double(lam[(long long)((1 + a) * Q + k) * P.plane + id]);
                mub[a] += k == 0 ? -(1.0 - w) * lh : w * lh;
            }
        }
        double phb = Gw;
        const double S0b = -0.5 * Gw;
        if (!P.source_off) {
            const double pp = interp_p(ph), dpp = interp_dp(ph);
            const double mu0[2] = {closure_dev(d[0], pp, 0, P), closure_dev(d[1], pp, 1, P)};
            const double dom = mu0[0] * P.dc[0] + mu0[1] * P.dc[1];
            const double B = -dwell_d(ph) + P.lam * dpp * dom;
            acc[4] += S0b * B;
            const double Bb = S0b * P.kphi;
            phb += Bb * (-dwell_dd(ph) + P.lam * interp_ddp(ph) * dom);
            const double domb = Bb * P.lam * dpp;
            mub[0] += domb * P.dc[0];
            mub[1] += domb * P.dc[1];
        }
        phb += -interp_dp(ph) * (P.dc[0] * mub[0] + P.dc[1] * mub[1]);
        phi0b[id] = phb;
    }
    block_accumulate(acc, partials, blockIdx.x, P, 0.0);
}

__global__ void theta_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double sm[kNTheta][256];
    for (int i = 0; i < kNTheta; ++i) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(long long)b * kNTheta + i];
        sm[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int i = 0; i < kNTheta; ++i) sm[i][threadIdx.x] += sm[i][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < kNTheta) out[threadIdx.x] = sm[threadIdx.x][0];
}

// ------------------------------------------------------------------------------------
template <class T, int LAT>
void adjoint_step_T(const DevParams& P, const StateView& st, bool odd, const void* lam_next, void* lam,
                    double* partials, cudaStream_t s) {
    using R = typename RealOf<T>::type;
    int bx;
    const dim3 grid = node_grid(P, bx);
    const double om_g_deriv = -P.om_g * P.om_g * P.inv_cs2;   // d om_g / d M_phi
    if (odd)
        adjoint_step_kernel<T, LAT, AA_ODD><<<grid, bx, 0, s>>>(P, st, static_cast<const R*>(lam_next),
                                                                static_cast<R*>(lam), partials, om_g_deriv);
    else
        adjoint_step_kernel<T, LAT, AA_EVEN><<<grid, bx, 0, s>>>(P, st, static_cast<const R*>(lam_next),
                                                                 static_cast<R*>(lam), partials, om_g_deriv);
}

template <class T, int LAT>
void adjoint_seed_T(const DevParams& P, const StateView& st, bool odd, const void* a, const void* b,
                    const void* c, void* lam, double* partials, cudaStream_t s) {
    using R = typename RealOf<T>::type;
    const R* pa = static_cast<const R*>(a);
    const R* pb = static_cast<const R*>(b);
    const R* pc = static_cast<const R*>(c);
    if (odd)
        adjoint_seed_kernel<T, LAT, AA_ODD><<<kAdjBlocks, 256, 0, s>>>(P, st, pa, pb, pc, static_cast<R*>(lam),
                                                                       partials);
    else
        adjoint_seed_kernel<T, LAT, AA_EVEN><<<kAdjBlocks, 256, 0, s>>>(P, st, pa, pb, pc, static_cast<R*>(lam),
                                                                        partials);
}

template <class T, int LAT>
void adjoint_init_T(const DevParams& P, const double* phi0, const double* cA0, const double* cB0, const void* lam,
                    double* phi0b, double* partials, cudaStream_t s) {
    using R = typename RealOf<T>::type;
    adjoint_init_kernel<T, LAT><<<kAdjBlocks, 256, 0, s>>>(P, phi0, cA0, cB0, static_cast<const R*>(lam), phi0b,
                                                           partials);
}

#define LBM_ADJ_DISPATCH(STORAGE, LAT, FN, ...)                                                 \
    do {                                                                                        \
        if (STORAGE == 0) {                                                                     \
            if (LAT == LAT_D2Q5) FN<double, LAT_D2Q5>(__VA_ARGS__);                             \
            else if (LAT == LAT_D2Q9) FN<double, LAT_D2Q9>(__VA_ARGS__);                        \
            else if (LAT == LAT_D3Q19) FN<double, LAT_D3Q19>(__VA_ARGS__);                      \
            else FN<double, LAT_D3Q7>(__VA_ARGS__);                                             \
        } else {                                                                                \
            if (LAT == LAT_D2Q5) FN<float, LAT_D2Q5>(__VA_ARGS__);                              \
            else if (LAT == LAT_D2Q9) FN<float, LAT_D2Q9>(__VA_ARGS__);                         \
            else if (LAT == LAT_D3Q19) FN<float, LAT_D3Q19>(__VA_ARGS__);                       \
            else FN<float, LAT_D3Q7>(__VA_ARGS__);                                              \
        }                                                                                       \
    } while (0)

void launch_adjoint_step(const DevParams& P, const StateView& st, int storage, int lat, bool odd,
                         const void* lam_next, void* lam, double* partials, cudaStream_t s) {
    LBM_ADJ_DISPATCH(storage, lat, adjoint_step_T, P, st, odd, lam_next, lam, partials, s);
}
void launch_adjoint_seed(const DevParams& P, const StateView& st, int storage, int lat, bool odd, const void* a,
                         const void* b, const void* c, void* lam, double* partials, cudaStream_t s) {
    LBM_ADJ_DISPATCH(storage, lat, adjoint_seed_T, P, st, odd, a, b, c, lam, partials, s);
}
void launch_adjoint_init(const DevParams& P, int storage, int lat, const double* phi0, const double* cA0,
                         const double* cB0, const void* lam, double* phi0b, double* partials, cudaStream_t s) {
    LBM_ADJ_DISPATCH(storage, lat, adjoint_init_T, P, phi0, cA0, cB0, lam, phi0b, partials, s);
}
void launch_theta_final(const double* partials, int rows, double* out, cudaStream_t s) {
    theta_final<<<1, 256, 0, s>>>(partials, rows, out);
}
// rows of FP64 partials: one per block of the step grid, at least one per block of the
// grid-stride seed and init kernels
long long adjoint_rows(const DevParams& P) {
    int bx;
    const dim3 g = node_grid(P, bx);
    const long long step_rows = (long long)g.x * g.y * g.z;
    return step_rows > kAdjBlocks ? step_rows : kAdjBlocks;
}
int adjoint_ntheta() { return kNTheta; }

}  // namespace lbm
