// C-ABI entry points (include/lbm.h): validation, buffer layout, launch sequencing.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_launch.h"

using lbm::DevParams;
using lbm::StateView;

namespace {

constexpr long long kAlign = 256;
constexpr int kRedBlocks = 1216;   // 152 SMs x 8 blocks of 256 threads

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

int scalar_q(int lattice) {
    return lattice == LBM_D2Q5 ? 5 : (lattice == LBM_D3Q19 ? 19 : (lattice == LBM_D2Q9 ? 9 : 7));
}
bool two_d(int lattice) { return lattice == LBM_D2Q5 || lattice == LBM_D2Q9; }
// the fused z-marching flow kernel is written for D3Q7 scalar sets
bool fused_flow(const lbm_params* p) { return p->flow && p->lattice == LBM_D3Q7; }
size_t storage_size(int s) { return s == LBM_F64 ? 8 : (s == LBM_F32 ? 4 : 2); }
bool is16(int s) { return s == LBM_F16 || s == LBM_BF16; }

thread_local std::string g_last_error = "no error";

struct Layout {
    long long n = 0, plane = 0;
    bool two = false;          // two state copies (fused pull step with flow)
    size_t copy = 0;           // bytes of one copy
    size_t state = 0, work = 0;
    size_t off_f = 0, off_g = 0, off_hA = 0, off_hB = 0, off_rest = 0;
    size_t off_phi = 0, off_bits = 0, off_partials = 0, off_out = 0;
    size_t off_phig[2] = {0, 0};   // slab: phi of the neighbours' edge planes (below, above)
};

const char* check_params(const lbm_params* p) {
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "lattice extents must be >= 1";
    if (p->ny > 65535 || p->nz > 65535) return "ny and nz must be <= 65535";
    if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return "nx*ny*nz must be < 2^31";
    if (p->lattice != LBM_D2Q5 && p->lattice != LBM_D3Q7 && p->lattice != LBM_D3Q19 && p->lattice != LBM_D2Q9)
        return "lattice must be LBM_D2Q5, LBM_D3Q7, LBM_D3Q19 or LBM_D2Q9";
    if (two_d(p->lattice) && p->nz != 1) return "the 2D lattices (LBM_D2Q5, LBM_D2Q9) need nz == 1";
    if (p->flow != 0 && p->flow != 1) return "flow must be 0 or 1";
    if (p->flow && two_d(p->lattice)) return "flow needs a 3D scalar lattice (LBM_D3Q7 or LBM_D3Q19)";
    if (p->storage < LBM_F64 || p->storage > LBM_BF16) return "storage must be one of lbm_storage";
    if (p->inplace != 0 && p->inplace != 1) return "inplace must be 0 or 1";
    if (!(p->W > 0)) return "W must be > 0";
    if (!(p->M_phi > 0)) return "M_phi must be > 0";
    for (int ph = 0; ph < 2; ++ph)
        for (int a = 0; a < 2; ++a)
            if (!(p->M[ph][a] > 0)) return "mobilities M must be > 0";
    if (p->flow && !(p->nu > 0)) return "nu must be > 0 with flow";
    if (!(p->f_scale == 0.0 || p->f_scale == 1024.0)) return "f_scale must be 0 or 1024 (the fixed 16-bit scale)";
    if (p->collision != LBM_BGK && p->collision != LBM_TRT && p->collision != LBM_MRT)
        return "collision must be LBM_BGK, LBM_TRT or LBM_MRT";
    for (int i = 0; i < 5; ++i)
        if (!(p->mrt_rates[i] >= 0 && p->mrt_rates[i] < 2)) return "mrt_rates must lie in [0, 2) (0 selects the default)";
    if (p->collision == LBM_TRT && !(p->trt_magic >= 0)) return "trt_magic must be >= 0 (0 selects 3/16)";
    return nullptr;
}

// slab: two state copies always, and two ghost phi planes in the work buffer
Layout layout_of(const lbm_params* p, bool slab = false) {
    Layout L;
    L.n = (long long)p->nx * p->ny * p->nz;
    L.plane = round_up(L.n, 128);
    const size_t es = storage_size(p->storage);
    const size_t pb = (size_t)L.plane * es;
    const int Q = scalar_q(p->lattice);
    size_t o = 0;
    L.off_f = o;  o += p->flow ? 19 * pb : 0;
    L.off_g = o;  o += Q * pb;
    L.off_hA = o; o += Q * pb;
    L.off_hB = o; o += Q * pb;
    // FP32 rest populations of 16-bit storage: g_0, hA_0, hB_0, f_0 (and f_0 of odd time levels
    // in place, see lbm::Addr)
    L.off_rest = o; o += is16(p->storage) ? 5 * (size_t)L.plane * sizeof(float) : 0;
    L.copy = round_up(o, kAlign);
    L.two = slab || (p->flow && !p->inplace);
    L.state = L.copy * (L.two ? 2 : 1);
    const size_t real = p->storage == LBM_F64 ? 8 : 4;
    size_t w = 0;
    // the phi field: read by the capillary stencil (flow) and by the 2D Euler count
    L.off_phi = w;      w += (p->flow || two_d(p->lattice)) ? round_up((size_t)L.plane * real, kAlign) : 0;
    // one bit per node of phi >= 1/2: the 3D Euler count
    L.off_bits = w;     w += two_d(p->lattice) ? 0 : round_up((size_t)((L.n + 31) / 32) * sizeof(unsigned), kAlign);
    L.off_partials = w; w += round_up((size_t)kRedBlocks * LBM_NRED * sizeof(double), kAlign);
    L.off_out = w;      w += round_up(LBM_NRED * sizeof(double), kAlign);
    for (int i = 0; i < 2; ++i) {
        L.off_phig[i] = w;
        w += slab ? round_up((size_t)p->nx * p->ny * real, kAlign) : 0;
    }
    L.work = w;
    return L;
}

template <class R>
void fill_coef(const DevParams& d, lbm::Coef<R>& c) {
    c.lam = R(d.lam);
    c.kphi = R(d.kphi);
    for (int a = 0; a < 2; ++a) {
        c.c0[a] = R(d.c0[a]);
        c.dc[a] = R(d.dc[a]);
        c.M0[a] = R(d.M0[a]);
        c.M1[a] = R(d.M1[a]);
    }
    c.om_g = R(d.om_g);
    c.om_f = R(d.om_f);
    c.om_fm = R(d.om_fm);
    for (int i = 0; i < 19; ++i) c.mrt[i] = R(d.mrt[i]);
    c.sw15 = R(d.sw15);
    c.inv_W2 = R(d.inv_W2);
    for (int i = 0; i < 3; ++i) c.g[i] = R(d.g[i]);
}

DevParams dev_params(const lbm_params* p, const Layout& L) {
    DevParams d{};
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    d.wall_x = p->wall_x != 0; d.wall_z = p->wall_z != 0; d.source_off = p->source_off != 0;
    d.wall_zlo = d.wall_zhi = d.wall_z;
    d.z_lo = 0;
    d.z_hi = p->nz;
    d.n = L.n; d.plane = L.plane;
    d.W = p->W; d.lam = p->lambda;
    d.kphi = p->M_phi / (p->W * p->W);
    const double cs2 = p->lattice == LBM_D3Q7 ? 0.25 : 1.0 / 3.0;
    d.inv_cs2 = 1.0 / cs2;
    for (int a = 0; a < 2; ++a) {
        d.c0[a] = p->c_eq[0][a];
        d.c1[a] = p->c_eq[1][a];
        d.dc[a] = p->c_eq[1][a] - p->c_eq[0][a];
        d.M0[a] = p->M[0][a];
        d.M1[a] = p->M[1][a];
    }
    d.om_g = 1.0 / (p->M_phi / cs2 + 0.5);
    d.om_f = p->flow ? 1.0 / (p->nu * 3.0 + 0.5) : 0.0;
    d.coll = p->flow ? p->collision : LBM_BGK;
    const double magic = p->trt_magic > 0 ? p->trt_magic : 3.0 / 16.0;
    d.om_fm = d.coll == LBM_TRT ? 1.0 / (magic / (p->nu * 3.0) + 0.5) : d.om_f;
    // MRT rates per moment: shear moments at om_f, the others from mrt_rates (0 = default)
    const double def[5] = {1.19, 1.4, 1.2, 1.4, 1.98};
    double r[5];
    for (int i = 0; i < 5; ++i) r[i] = p->mrt_rates[i] > 0 ? p->mrt_rates[i] : def[i];
    const double rate[19] = {d.om_f, r[0], r[1], d.om_f, r[2], d.om_f, r[2], d.om_f, r[2], d.om_f, r[3],
                             d.om_f, r[3], d.om_f, d.om_f, d.om_f, r[4], r[4], r[4]};
    for (int i = 0; i < 19; ++i) d.mrt[i] = rate[i] / lbm::MRT19::norm(i);
    d.sw15 = 1.5 * p->sigma * p->W;
    d.inv_W2 = 1.0 / (p->W * p->W);
    for (int i = 0; i < 3; ++i) d.g[i] = p->g[i];
    d.f_scale = p->f_scale > 0 ? p->f_scale : 1024.0;
    d.inv_f_scale = 1.0 / d.f_scale;
    fill_coef(d, d.cd);
    fill_coef(d, d.cf);
    return d;
}

}  // namespace

struct lbm_ctx {
    lbm_params p;
    Layout L;
    DevParams dp;
    StateView st;                  // copy 0 (the only copy for the in-place layout)
    StateView st1;                 // copy 1 of the two-buffer layout
    char* work;
    cudaStream_t stream;
    int64_t t;
    std::string err;
    std::vector<cudaEvent_t> ev;   // profiling: 3 events per timed step
    int prof_max = 0, prof_n = 0;
    cudaGraphExec_t graph = nullptr;   // two steps captured from an even time level
    // slab of a z-decomposed lattice (lbm_slab_init): global first plane, own planes, and
    // whether a neighbour's plane sits below / above (ghost planes z_lo - 1 and z_hi)
    bool slab = false;
    int z0 = 0, nzl = 0, glo = 0, ghi = 0;
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
    if (c) c->err = msg; else g_last_error = msg;
    return s;
}

lbm_status cuda_check(lbm_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LBM_OK;
}

#define LBM_DISPATCH(STORAGE, FN, ...)                                         \
    switch (STORAGE) {                                                         \
        case LBM_F64: lbm::FN##_f64(__VA_ARGS__); break;                       \
        case LBM_F32: lbm::FN##_f32(__VA_ARGS__); break;                       \
        case LBM_F16: lbm::FN##_f16(__VA_ARGS__); break;                       \
        default: lbm::FN##_bf16(__VA_ARGS__); break;                           \
    }

__global__ void reduce_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double sm[LBM_NRED][256];
    for (int i = 0; i < LBM_NRED; ++i) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            double u = partials[(long long)b * LBM_NRED + i];
            v = (i == LBM_RED_UMAX) ? fmax(v, u) : v + u;
        }
        sm[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int i = 0; i < LBM_NRED; ++i)
                sm[i][threadIdx.x] = (i == LBM_RED_UMAX) ? fmax(sm[i][threadIdx.x], sm[i][threadIdx.x + s])
                                                         : sm[i][threadIdx.x] + sm[i][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < LBM_NRED) out[threadIdx.x] = sm[threadIdx.x][0];
}

// Views of one state copy starting at base, with the pointer of every population plane.
StateView view_of(const lbm_params* p, const Layout& L, void* base) {
    StateView v{};
    char* s = static_cast<char*>(base);
    const size_t pb = (size_t)L.plane * storage_size(p->storage);
    const int Q = scalar_q(p->lattice);
    v.f = p->flow ? s + L.off_f : nullptr;
    v.g = s + L.off_g;
    v.hA = s + L.off_hA;
    v.hB = s + L.off_hB;
    v.rest = is16(p->storage) ? reinterpret_cast<float*>(s + L.off_rest) : nullptr;
    for (int k = 0; k < 19; ++k) v.plane[k] = p->flow ? s + L.off_f + k * pb : nullptr;
    for (int k = 0; k < Q; ++k) {
        v.plane[19 + k] = s + L.off_g + k * pb;              // Planes<LAT>::G, HA, HB
        v.plane[19 + Q + k] = s + L.off_hA + k * pb;
        v.plane[19 + 2 * Q + k] = s + L.off_hB + k * pb;
    }
    return v;
}

lbm_status bind(const lbm_params* p, void* d_state, void* d_work, void* stream, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (const char* m = check_params(p)) return fail(nullptr, LBM_ERR_ARG, m);
    if (!d_state || !d_work) return fail(nullptr, LBM_ERR_ARG, "state and work buffers must be non-NULL");
    if (((uintptr_t)d_state % kAlign) || ((uintptr_t)d_work % kAlign))
        return fail(nullptr, LBM_ERR_ARG, "state and work buffers must be 256-byte aligned");
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_ARG, "host allocation of the context failed");
    c->p = *p;
    c->L = layout_of(p);
    c->dp = dev_params(p, c->L);
    c->st = view_of(p, c->L, d_state);
    c->st1 = c->L.two ? view_of(p, c->L, static_cast<char*>(d_state) + c->L.copy) : c->st;
    c->work = static_cast<char*>(d_work);
    c->stream = static_cast<cudaStream_t>(stream);
    c->t = 0;
    c->err = "no error";
    *out = c;
    return LBM_OK;
}

// State view holding time level t and the streaming mode that reads it.
const StateView& current(const lbm_ctx* c) { return (c->L.two && (c->t & 1)) ? c->st1 : c->st; }
int read_mode(const lbm_ctx* c) {
    if (c->L.two) return lbm::kModePull;
    return (c->t & 1) ? lbm::kModeAAOdd : lbm::kModeAAEven;
}
// z planes one block of the fused flow kernel marches through (measured best of 16..128 at 512^3)
constexpr int kZChunk = 32;
int zchunk_of(const lbm_params* p) { return p->nz < kZChunk ? p->nz : kZChunk; }

}  // namespace

extern "C" {

size_t lbm_state_bytes(const lbm_params* p) {
    if (check_params(p)) return 0;
    return layout_of(p).state;
}

size_t lbm_work_bytes(const lbm_params* p) {
    if (check_params(p)) return 0;
    return layout_of(p).work;
}

lbm_status lbm_init(const lbm_params* p, void* d_state, void* d_work, const double* d_phi0,
                    const double* d_cA0, const double* d_cB0, void* stream, lbm_ctx** out) {
    if (!d_phi0 || !d_cA0 || !d_cB0) {
        if (out) *out = nullptr;
        return fail(nullptr, LBM_ERR_ARG, "initial fields must be non-NULL device pointers");
    }
    lbm_status s = bind(p, d_state, d_work, stream, out);
    if (s != LBM_OK) return s;
    lbm_ctx* c = *out;
    cudaGetLastError();
    LBM_DISPATCH(c->p.storage, launch_init, c->dp, c->st, c->p.lattice, c->p.flow != 0, c->L.two, d_phi0, d_cA0,
                 d_cB0, c->stream);
    s = cuda_check(c, "init kernel launch");
    if (s != LBM_OK) {
        g_last_error = c->err;
        delete c;
        *out = nullptr;
    }
    return s;
}

lbm_status lbm_attach(const lbm_params* p, void* d_state, void* d_work, int64_t t, void* stream, lbm_ctx** out) {
    if (t < 0) {
        if (out) *out = nullptr;
        return fail(nullptr, LBM_ERR_ARG, "t must be >= 0");
    }
    lbm_status s = bind(p, d_state, d_work, stream, out);
    if (s == LBM_OK) (*out)->t = t;
    return s;
}

namespace {
// Slab: copy the neighbours' edge-plane phi (received by lbm_slab_phi_unpack) into the phi
// field's planes z_lo - 1 and z_hi, where the per-node kernels' stencil reads it.
void ghost_phi_to_field(lbm_ctx* c) {
    const size_t real = c->p.storage == LBM_F64 ? 8 : 4;
    const size_t pb = (size_t)c->p.nx * c->p.ny * real;
    char* phi = c->work + c->L.off_phi;
    if (c->glo) cudaMemcpyAsync(phi + (size_t)(c->dp.z_lo - 1) * pb, c->work + c->L.off_phig[0], pb,
                                cudaMemcpyDeviceToDevice, c->stream);
    if (c->ghi) cudaMemcpyAsync(phi + (size_t)c->dp.z_hi * pb, c->work + c->L.off_phig[1], pb,
                                cudaMemcpyDeviceToDevice, c->stream);
}

// Queue the kernels that advance time level t to t + 1 (no change to the context).
void launch_one(lbm_ctx* c, int64_t t, cudaEvent_t* e) {
    const int mode = c->L.two ? lbm::kModePull : ((t & 1) ? lbm::kModeAAOdd : lbm::kModeAAEven);
    if (e) cudaEventRecord(e[0], c->stream);
    // src holds time level t; dst receives t + 1 (the same buffer in the in-place layout)
    const StateView& src = (c->L.two && (t & 1)) ? c->st1 : c->st;
    const StateView& dst = c->L.two ? ((t & 1) ? c->st : c->st1) : c->st;
    const bool fused = c->L.two && fused_flow(&c->p);
    if (c->p.flow && !fused) {
        LBM_DISPATCH(c->p.storage, launch_phi, c->dp, src, c->p.lattice, mode, c->work + c->L.off_phi, c->stream);
        if (c->slab) ghost_phi_to_field(c);
    }
    if (e) cudaEventRecord(e[1], c->stream);
    if (fused) {
        LBM_DISPATCH(c->p.storage, launch_fused, c->dp, src, dst, zchunk_of(&c->p), c->stream);
    } else {
        LBM_DISPATCH(c->p.storage, launch_step, c->dp, src, dst, c->p.lattice, c->p.flow != 0, mode,
                     c->work + c->L.off_phi, c->stream);
    }
    if (e) cudaEventRecord(e[2], c->stream);
}
}  // namespace

lbm_status lbm_step(lbm_ctx* c, int nsteps) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps must be >= 0");
    if (c->slab && nsteps > 1)
        return fail(c, LBM_ERR_STATE, "a slab advances one step per call: exchange its halos between steps");
    cudaGetLastError();
    for (int i = 0; i < nsteps; ++i) {
        const bool timed = c->prof_n < c->prof_max;
        launch_one(c, c->t, timed ? &c->ev[3 * c->prof_n] : nullptr);
        if (timed) c->prof_n += 1;
        c->t += 1;
    }
    return cuda_check(c, "step kernel launch");
}

lbm_status lbm_step_graph(lbm_ctx* c, int nsteps) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps must be >= 0");
    if (c->stream == nullptr || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread)
        return fail(c, LBM_ERR_ARG, "graph replay needs a created (capturable) stream, not a default stream");
    if (c->slab) return fail(c, LBM_ERR_STATE, "graph replay of two steps does not apply to a slab");
    if (nsteps == 0) return LBM_OK;
    if (c->t & 1) {                                  // align to an even time level
        lbm_status s = lbm_step(c, 1);
        if (s != LBM_OK || --nsteps == 0) return s;
    }
    if (!c->graph && nsteps >= 2) {
        // one plain pair of steps first: every kernel's one-time set-up happens outside capture
        lbm_status s = lbm_step(c, 2);
        if (s != LBM_OK) return s;
        nsteps -= 2;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            launch_one(c, c->t, nullptr);
            launch_one(c, c->t + 1, nullptr);
            e = cudaStreamEndCapture(c->stream, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            cudaGetLastError();
            return fail(c, LBM_ERR_CUDA, std::string("step graph capture: ") + cudaGetErrorString(e));
        }
    }
    for (; nsteps >= 2; nsteps -= 2) {
        cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
        if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("step graph launch: ") + cudaGetErrorString(e));
        c->t += 2;
    }
    return nsteps ? lbm_step(c, 1) : cuda_check(c, "step graph");
}

lbm_status lbm_profile_begin(lbm_ctx* c, int max_steps) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (max_steps < 0 || max_steps > 1000000) return fail(c, LBM_ERR_ARG, "max_steps out of range");
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.assign(3 * (size_t)max_steps, nullptr);
    for (auto& e : c->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            c->prof_max = c->prof_n = 0;
            return cuda_check(c, "profile event create");
        }
    }
    c->prof_max = max_steps;
    c->prof_n = 0;
    return LBM_OK;
}

lbm_status lbm_profile_end(lbm_ctx* c, double* out) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    cudaError_t err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("profile sync: ") + cudaGetErrorString(err));
    double a = 0.0, b = 0.0;
    for (int i = 0; i < c->prof_n; ++i) {
        float m0 = 0.f, m1 = 0.f;
        cudaEventElapsedTime(&m0, c->ev[3 * i], c->ev[3 * i + 1]);
        cudaEventElapsedTime(&m1, c->ev[3 * i + 1], c->ev[3 * i + 2]);
        a += m0;
        b += m1;
    }
    out[0] = a; out[1] = b; out[2] = c->prof_n;
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    c->prof_max = c->prof_n = 0;
    return cuda_check(c, "profile events");
}

int lbm_kernels_per_step(const lbm_ctx* c) {
    return c ? ((c->p.flow && !(c->L.two && fused_flow(&c->p))) ? 2 : 1) : 0;
}

int64_t lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

lbm_status lbm_fields(lbm_ctx* c, void* const* dst) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!dst) return fail(c, LBM_ERR_ARG, "dst is NULL");
    lbm::FieldPtrs fp;
    for (int i = 0; i < LBM_NFIELDS; ++i) fp.p[i] = dst[i];
    cudaGetLastError();
    if (c->slab && c->p.flow) ghost_phi_to_field(c);
    LBM_DISPATCH(c->p.storage, launch_fields, c->dp, current(c), c->p.lattice, c->p.flow != 0, read_mode(c),
                 c->work + c->L.off_phi, fp, c->stream);
    return cuda_check(c, "fields kernel launch");
}

lbm_status lbm_reduce(lbm_ctx* c, double* out) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    cudaGetLastError();
    double* partials = reinterpret_cast<double*>(c->work + c->L.off_partials);
    double* dout = reinterpret_cast<double*>(c->work + c->L.off_out);
    if (c->slab && c->p.flow) ghost_phi_to_field(c);
    // a slab keeps no bit field: its droplet count (LBM_RED_EULER) is left at 0
    LBM_DISPATCH(c->p.storage, launch_reduce, c->dp, current(c), c->p.lattice, c->p.flow != 0, read_mode(c),
                 c->work + c->L.off_phi, c->slab ? nullptr : c->work + c->L.off_bits, partials, kRedBlocks,
                 c->stream);
    reduce_final<<<1, 256, 0, c->stream>>>(partials, kRedBlocks, dout);
    lbm_status s = cuda_check(c, "reduce kernel launch");
    if (s != LBM_OK) return s;
    cudaError_t e = cudaMemcpyAsync(out, dout, LBM_NRED * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("reduce copy: ") + cudaGetErrorString(e));
    if (out[LBM_RED_NONFINITE] != 0.0)
        return fail(c, LBM_ERR_UNSTABLE, "non-finite moments in the state (unstable run)");
    return LBM_OK;
}

size_t lbm_copy_bytes(const lbm_params* p) {
    if (check_params(p)) return 0;
    return layout_of(p).copy;
}

lbm_status lbm_step_buffers(const lbm_params* p, const void* d_src, void* d_dst, int64_t t, void* d_work,
                            void* stream) {
    if (const char* m = check_params(p)) return fail(nullptr, LBM_ERR_ARG, m);
    if (!d_src || !d_dst || t < 0) return fail(nullptr, LBM_ERR_ARG, "buffers must be non-NULL and t >= 0");
    if (d_src == d_dst) return fail(nullptr, LBM_ERR_ARG, "d_src and d_dst must differ");
    const Layout L = layout_of(p);
    if (p->flow && !(L.two && fused_flow(p)) && !d_work) return fail(nullptr, LBM_ERR_ARG, "this flow step needs d_work (phi pass)");
    const DevParams dp = dev_params(p, L);
    const StateView src = view_of(p, L, const_cast<void*>(d_src));
    const StateView dst = view_of(p, L, d_dst);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    if (L.two && fused_flow(p)) {
        LBM_DISPATCH(p->storage, launch_fused, dp, src, dst, zchunk_of(p), s);
    } else {
        const int mode = L.two ? lbm::kModePull : ((t & 1) ? lbm::kModeAAOdd : lbm::kModeAAEven);
        char* phi = static_cast<char*>(d_work) + L.off_phi;
        if (p->flow) { LBM_DISPATCH(p->storage, launch_phi, dp, src, p->lattice, mode, phi, s); }
        LBM_DISPATCH(p->storage, launch_step, dp, src, dst, p->lattice, p->flow != 0, mode, phi, s);
    }
    return cuda_check(nullptr, "step_buffers kernel launch");
}

namespace {
const char* check_adjoint(const lbm_params* p) {
    if (const char* m = check_params(p)) return m;
    if (p->flow) return "the adjoint covers the step without flow";
    if (p->storage != LBM_F32 && p->storage != LBM_F64) return "the adjoint needs LBM_F32 or LBM_F64 storage";
    return nullptr;
}
size_t real_size(const lbm_params* p) { return p->storage == LBM_F64 ? 8 : 4; }
}  // namespace

size_t lbm_adjoint_bytes(const lbm_params* p) {
    if (check_adjoint(p)) return 0;
    return round_up(3 * (size_t)scalar_q(p->lattice) * layout_of(p).plane * real_size(p), kAlign);
}

size_t lbm_adjoint_work_bytes(const lbm_params* p) {
    if (check_adjoint(p)) return 0;
    const long long rows = lbm::adjoint_rows(dev_params(p, layout_of(p)));
    return round_up((size_t)(rows + 1) * lbm::adjoint_ntheta() * sizeof(double), kAlign);
}

lbm_status lbm_adjoint_reset(const lbm_params* p, void* d_adj_work, void* stream) {
    if (const char* m = check_adjoint(p)) return fail(nullptr, check_params(p) ? LBM_ERR_ARG : LBM_ERR_STATE, m);
    if (!d_adj_work) return fail(nullptr, LBM_ERR_ARG, "d_adj_work is NULL");
    cudaError_t e = cudaMemsetAsync(d_adj_work, 0, lbm_adjoint_work_bytes(p), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, std::string("adjoint reset: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_adjoint_seed(const lbm_params* p, const void* d_state, int64_t t, const void* d_phib,
                            const void* d_muAb, const void* d_muBb, void* d_lam, void* d_adj_work, void* stream) {
    if (const char* m = check_adjoint(p)) return fail(nullptr, check_params(p) ? LBM_ERR_ARG : LBM_ERR_STATE, m);
    if (!d_state || !d_lam || !d_adj_work || t < 0) return fail(nullptr, LBM_ERR_ARG, "NULL buffer or t < 0");
    const Layout L = layout_of(p);
    cudaGetLastError();
    lbm::launch_adjoint_seed(dev_params(p, L), view_of(p, L, const_cast<void*>(d_state)), p->storage, p->lattice,
                             (t & 1) != 0, d_phib, d_muAb, d_muBb, d_lam, static_cast<double*>(d_adj_work),
                             static_cast<cudaStream_t>(stream));
    return cuda_check(nullptr, "adjoint seed launch");
}

lbm_status lbm_adjoint_step(const lbm_params* p, const void* d_state, int64_t t, const void* d_lam_next,
                            void* d_lam, void* d_adj_work, void* stream) {
    if (const char* m = check_adjoint(p)) return fail(nullptr, check_params(p) ? LBM_ERR_ARG : LBM_ERR_STATE, m);
    if (!d_state || !d_lam || !d_lam_next || !d_adj_work || t < 0)
        return fail(nullptr, LBM_ERR_ARG, "NULL buffer or t < 0");
    if (d_lam == d_lam_next) return fail(nullptr, LBM_ERR_ARG, "d_lam and d_lam_next must differ");
    const Layout L = layout_of(p);
    cudaGetLastError();
    lbm::launch_adjoint_step(dev_params(p, L), view_of(p, L, const_cast<void*>(d_state)), p->storage, p->lattice,
                             (t & 1) != 0, d_lam_next, d_lam, static_cast<double*>(d_adj_work),
                             static_cast<cudaStream_t>(stream));
    return cuda_check(nullptr, "adjoint step launch");
}

lbm_status lbm_adjoint_segment(const lbm_params* p, void* d_ring, int64_t t0, int n, void* d_lam, void* d_lam_tmp,
                               void* d_adj_work, void* d_work, void* stream, int* which) {
    if (const char* m = check_adjoint(p)) return fail(nullptr, check_params(p) ? LBM_ERR_ARG : LBM_ERR_STATE, m);
    if (!d_ring || !d_lam || !d_lam_tmp || !d_adj_work || !which || t0 < 0 || n < 1)
        return fail(nullptr, LBM_ERR_ARG, "NULL buffer, t0 < 0 or n < 1");
    const Layout L = layout_of(p);
    char* ring = static_cast<char*>(d_ring);
    for (int j = 1; j < n; ++j) {
        lbm_status s = lbm_step_buffers(p, ring + (j - 1) * L.copy, ring + j * L.copy, t0 + j - 1, d_work, stream);
        if (s != LBM_OK) return s;
    }
    void* cur = d_lam;
    void* nxt = d_lam_tmp;
    for (int j = n - 1; j >= 0; --j) {
        lbm_status s = lbm_adjoint_step(p, ring + j * L.copy, t0 + j, cur, nxt, d_adj_work, stream);
        if (s != LBM_OK) return s;
        void* t = cur; cur = nxt; nxt = t;
    }
    *which = cur == d_lam ? 0 : 1;
    return LBM_OK;
}

lbm_status lbm_adjoint_init(const lbm_params* p, const double* d_phi0, const double* d_cA0, const double* d_cB0,
                            const void* d_lam0, double* d_phi0b, void* d_adj_work, void* stream) {
    if (const char* m = check_adjoint(p)) return fail(nullptr, check_params(p) ? LBM_ERR_ARG : LBM_ERR_STATE, m);
    if (!d_phi0 || !d_cA0 || !d_cB0 || !d_lam0 || !d_phi0b || !d_adj_work)
        return fail(nullptr, LBM_ERR_ARG, "NULL buffer");
    const Layout L = layout_of(p);
    cudaGetLastError();
    lbm::launch_adjoint_init(dev_params(p, L), p->storage, p->lattice, d_phi0, d_cA0, d_cB0, d_lam0, d_phi0b,
                             static_cast<double*>(d_adj_work), static_cast<cudaStream_t>(stream));
    return cuda_check(nullptr, "adjoint init launch");
}

lbm_status lbm_adjoint_theta(const lbm_params* p, void* d_adj_work, double* out, void* stream) {
    if (const char* m = check_adjoint(p)) return fail(nullptr, check_params(p) ? LBM_ERR_ARG : LBM_ERR_STATE, m);
    if (!d_adj_work || !out) return fail(nullptr, LBM_ERR_ARG, "NULL buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* partials = static_cast<double*>(d_adj_work);
    const long long rows = lbm::adjoint_rows(dev_params(p, layout_of(p)));
    double* dout = partials + (size_t)rows * lbm::adjoint_ntheta();
    cudaGetLastError();
    lbm::launch_theta_final(partials, int(rows), dout, s);
    lbm_status st = cuda_check(nullptr, "adjoint theta launch");
    if (st != LBM_OK) return st;
    cudaError_t e = cudaMemcpyAsync(out, dout, lbm::adjoint_ntheta() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, std::string("adjoint theta copy: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Slabs of a lattice decomposed along z (the paper's domain decomposition, §3).
namespace {

const char* check_slab(const lbm_params* p, int z0, int nzl) {
    if (const char* m = check_params(p)) return m;
    if (two_d(p->lattice)) return "slabs split a 3D lattice along z";
    if (p->inplace) return "slabs use the two-buffer layout (inplace must be 0)";
    if (z0 < 0 || nzl < 1 || (long long)z0 + nzl > p->nz) return "slab planes [z0, z0 + nzl) must lie in [0, nz)";
    return nullptr;
}

// The slab's own lattice: its planes plus one ghost plane on each side that has a
// neighbour (another slab, or the slab itself across a periodic end).
lbm_params slab_lattice(const lbm_params* p, int z0, int nzl, int& glo, int& ghi) {
    glo = (z0 > 0 || !p->wall_z) ? 1 : 0;
    ghi = (z0 + nzl < p->nz || !p->wall_z) ? 1 : 0;
    lbm_params q = *p;
    q.nz = nzl + glo + ghi;
    return q;
}

// Slot planes of one set whose velocity has z component ez (in the lattice's order).
template <class Lat>
void slots_with_ez(int Q, int ez, int first, std::vector<int>& out) {
    for (int k = 1; k < Q; ++k)
        if (Lat::ez(k) == ez) out.push_back(first + k);
}

// Pieces of one face message: (population plane, element size); -1 stands for the FP32 f_0
// plane of 16-bit storage, the reference of the moving f (Codec16Pop).
std::vector<int> face_planes(const lbm_params* p, int ez) {
    std::vector<int> v;
    if (p->flow) slots_with_ez<lbm::D3Q19>(19, ez, 0, v);
    const int Q = scalar_q(p->lattice);
    for (int set = 0; set < 3; ++set) {
        if (p->lattice == LBM_D3Q19) slots_with_ez<lbm::Scalar<lbm::LAT_D3Q19>>(Q, ez, 19 + set * Q, v);
        else slots_with_ez<lbm::Scalar<lbm::LAT_D3Q7>>(Q, ez, 19 + set * Q, v);
    }
    if (p->flow && is16(p->storage)) v.push_back(-1);
    return v;
}

size_t face_bytes(const lbm_params* p) {
    const size_t nxy = (size_t)p->nx * p->ny;
    size_t b = 0;
    for (int k : face_planes(p, 1)) b += nxy * (k < 0 ? sizeof(float) : storage_size(p->storage));
    return b;
}

// Copy plane z of every piece between the state copy st and a packed message.
lbm_status face_copy(lbm_ctx* c, const StateView& st, int ez, int z, void* msg, bool pack) {
    const size_t nxy = (size_t)c->p.nx * c->p.ny;
    const size_t es = storage_size(c->p.storage);
    char* m = static_cast<char*>(msg);
    for (int k : face_planes(&c->p, ez)) {
        const size_t eb = k < 0 ? sizeof(float) : es;
        char* plane = k < 0 ? reinterpret_cast<char*>(st.rest + 3 * c->L.plane) : static_cast<char*>(st.plane[k]);
        char* at = plane + (size_t)z * nxy * eb;
        cudaError_t e = pack ? cudaMemcpyAsync(m, at, nxy * eb, cudaMemcpyDeviceToDevice, c->stream)
                             : cudaMemcpyAsync(at, m, nxy * eb, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("slab halo copy: ") + cudaGetErrorString(e));
        m += nxy * eb;
    }
    return LBM_OK;
}

lbm_status check_side(lbm_ctx* c, int side, const void* buf) {
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!c->slab) return fail(c, LBM_ERR_STATE, "not a slab context (lbm_slab_init)");
    if (side != 0 && side != 1) return fail(c, LBM_ERR_ARG, "side must be 0 (below) or 1 (above)");
    if (!buf) return fail(c, LBM_ERR_ARG, "message buffer is NULL");
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_slab_state_bytes(const lbm_params* p, int32_t z0, int32_t nzl) {
    if (check_slab(p, z0, nzl)) return 0;
    int glo, ghi;
    const lbm_params q = slab_lattice(p, z0, nzl, glo, ghi);
    return layout_of(&q, true).state;
}

size_t lbm_slab_work_bytes(const lbm_params* p, int32_t z0, int32_t nzl) {
    if (check_slab(p, z0, nzl)) return 0;
    int glo, ghi;
    const lbm_params q = slab_lattice(p, z0, nzl, glo, ghi);
    return layout_of(&q, true).work;
}

int32_t lbm_slab_planes(const lbm_params* p, int32_t z0, int32_t nzl) {
    if (check_slab(p, z0, nzl)) return 0;
    int glo, ghi;
    return slab_lattice(p, z0, nzl, glo, ghi).nz;
}

lbm_status lbm_slab_init(const lbm_params* p, int32_t z0, int32_t nzl, void* d_state, void* d_work,
                         const double* d_phi0, const double* d_cA0, const double* d_cB0, void* stream,
                         lbm_ctx** out) {
    if (out) *out = nullptr;
    if (const char* m = check_slab(p, z0, nzl)) return fail(nullptr, LBM_ERR_ARG, m);
    if (!d_phi0 || !d_cA0 || !d_cB0) return fail(nullptr, LBM_ERR_ARG, "initial fields must be non-NULL device pointers");
    int glo, ghi;
    const lbm_params q = slab_lattice(p, z0, nzl, glo, ghi);
    lbm_status s = bind(&q, d_state, d_work, stream, out);
    if (s != LBM_OK) return s;
    lbm_ctx* c = *out;
    c->slab = true;
    c->z0 = z0; c->nzl = nzl; c->glo = glo; c->ghi = ghi;
    c->L = layout_of(&q, true);
    c->dp = dev_params(&q, c->L);
    c->dp.wall_zlo = p->wall_z && z0 == 0;
    c->dp.wall_zhi = p->wall_z && z0 + nzl == p->nz;
    c->dp.z_lo = glo;
    c->dp.z_hi = glo + nzl;
    c->dp.phi_ghost[0] = glo ? c->work + c->L.off_phig[0] : nullptr;
    c->dp.phi_ghost[1] = ghi ? c->work + c->L.off_phig[1] : nullptr;
    c->st = view_of(&q, c->L, d_state);
    c->st1 = view_of(&q, c->L, static_cast<char*>(d_state) + c->L.copy);
    cudaGetLastError();
    if (is16(q.storage) && q.flow) {
        // the ghost planes' f_0 is the reference of the populations init places there (0)
        const size_t pb = (size_t)q.nx * q.ny * sizeof(float);
        for (const StateView* v : {&c->st, &c->st1}) {
            char* f0 = reinterpret_cast<char*>(v->rest + 3 * c->L.plane);
            if (glo) cudaMemsetAsync(f0 + (size_t)(glo - 1) * pb, 0, pb, c->stream);
            if (ghi) cudaMemsetAsync(f0 + (size_t)(glo + nzl) * pb, 0, pb, c->stream);
        }
    }
    LBM_DISPATCH(q.storage, launch_init, c->dp, c->st, q.lattice, q.flow != 0, true, d_phi0, d_cA0, d_cB0, c->stream);
    s = cuda_check(c, "slab init kernel launch");
    if (s != LBM_OK) {
        g_last_error = c->err;
        delete c;
        *out = nullptr;
    }
    return s;
}

size_t lbm_slab_halo_bytes(const lbm_ctx* c) { return (c && c->slab) ? face_bytes(&c->p) : 0; }

size_t lbm_slab_phi_bytes(const lbm_ctx* c) {
    return (c && c->slab) ? (size_t)c->p.nx * c->p.ny * (c->p.storage == LBM_F64 ? 8 : 4) : 0;
}

lbm_status lbm_slab_pack(lbm_ctx* c, int32_t side, void* d_msg) {
    if (lbm_status s = check_side(c, side, d_msg)) return s;
    // side 0: the lowest own plane's populations moving down; side 1: the highest's moving up
    return face_copy(c, current(c), side ? 1 : -1, side ? c->dp.z_hi - 1 : c->dp.z_lo, d_msg, true);
}

lbm_status lbm_slab_unpack(lbm_ctx* c, int32_t side, const void* d_msg) {
    if (lbm_status s = check_side(c, side, d_msg)) return s;
    if (!(side ? c->ghi : c->glo)) return fail(c, LBM_ERR_STATE, "no neighbour on that side (wall)");
    // ghost below receives the lower neighbour's upward populations, ghost above the downward
    return face_copy(c, current(c), side ? -1 : 1, side ? c->dp.z_hi : c->dp.z_lo - 1, const_cast<void*>(d_msg),
                     false);
}

lbm_status lbm_slab_phi_pack(lbm_ctx* c, int32_t side, void* d_phi) {
    if (lbm_status s = check_side(c, side, d_phi)) return s;
    cudaGetLastError();
    LBM_DISPATCH(c->p.storage, launch_plane_phi, c->dp, current(c), c->p.lattice, lbm::kModePull,
                 side ? c->dp.z_hi - 1 : c->dp.z_lo, d_phi, c->stream);
    return cuda_check(c, "slab phi kernel launch");
}

lbm_status lbm_slab_phi_unpack(lbm_ctx* c, int32_t side, const void* d_phi) {
    if (lbm_status s = check_side(c, side, d_phi)) return s;
    if (!(side ? c->ghi : c->glo)) return fail(c, LBM_ERR_STATE, "no neighbour on that side (wall)");
    cudaError_t e = cudaMemcpyAsync(c->work + c->L.off_phig[side], d_phi, lbm_slab_phi_bytes(c),
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, LBM_ERR_CUDA, std::string("slab phi copy: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int32_t lbm_slab_ghosts(const lbm_ctx* c) { return (c && c->slab) ? (c->glo | (c->ghi << 1)) : -1; }

lbm_status lbm_destroy(lbm_ctx* c) {
    if (c) for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c && c->graph) cudaGraphExecDestroy(c->graph);
    delete c;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) {
    return c ? c->err.c_str() : g_last_error.c_str();
}

double lbm_mean_radius(const lbm_params* p, const double* sums) {
    if (!p || !sums) return NAN;
    const double n = sums[LBM_RED_EULER], a = sums[LBM_RED_INTERFACE];
    if (!(n > 0)) return NAN;
    const double pi = 3.14159265358979323846;
    return two_d(p->lattice) ? a / (2.0 * pi * n) : sqrt(a / (4.0 * pi * n));
}

const char* lbm_build_info(void) {
    return "gplbm sm_103a: fused collide-stream (AA in place; two-buffer z-marching with flow); "
           "storage f64/f32/f16 (fixed-point g; FP16 f, h; f against its writer's f_0)/bf16; scalar lattices "
           "D2Q5/D2Q9/D3Q7/D3Q19, flow D3Q19 BGK/TRT/MRT; adjoint";
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Allocation-free variant of lbm_reduce (see include/lbm.h): its scratch lives in this
// file-scope device array instead of the caller's work buffer.
namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device. In host code the array's name
// only stands in for the symbol, so the address is looked up with that device current. The
// lookup is repeated on every call (a host-side query once the module is loaded), so a
// device reset between calls cannot leave a stale address behind.
lbm_status static_scratch(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
        return fail(nullptr, LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return LBM_OK;
}

// The state buffer and the stream must belong to the current device, whose copy of the
// array the kernels are given.
lbm_status check_static_device(const void* d_state, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    cudaPointerAttributes a{};
    e = cudaPointerGetAttributes(&a, d_state);
    if (e != cudaSuccess || a.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(nullptr, LBM_ERR_ARG, "lbm_reduce_static: d_state is not device memory");
    }
    if (a.device != dev) return fail(nullptr, LBM_ERR_ARG, "lbm_reduce_static: d_state lies on another device than the current one");
    int sdev = dev;
    e = cudaStreamGetDevice(s, &sdev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, LBM_ERR_ARG, "lbm_reduce_static: invalid stream");
    }
    if (sdev != dev) return fail(nullptr, LBM_ERR_ARG, "lbm_reduce_static: the stream belongs to another device than the current one");
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_reduce_static(const lbm_params* p, const void* d_state, int64_t t, double* out,
                                        void* stream) {
    if (const char* m = check_params(p)) return fail(nullptr, LBM_ERR_ARG, m);
    if (!d_state || !out || t < 0) return fail(nullptr, LBM_ERR_ARG, "d_state and out must be non-NULL, t >= 0");
    if ((uintptr_t)d_state % kAlign) return fail(nullptr, LBM_ERR_ARG, "d_state must be 256-byte aligned");
    const Layout L = layout_of(p);
    if (L.work > kStaticScratchBytes)
        return fail(nullptr, LBM_ERR_ARG,
                    "lbm_reduce_static: this lattice needs " + std::to_string(L.work) +
                        " bytes of scratch (phi field, bit field and partials) but the static array holds " +
                        std::to_string(kStaticScratchBytes) + "; use lbm_reduce with a work buffer");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    lbm_status s = check_static_device(d_state, cs);
    if (s != LBM_OK) return s;
    void* scratch = nullptr;
    s = static_scratch(&scratch);
    if (s != LBM_OK) return s;
    char* w = static_cast<char*>(scratch);
    const DevParams dp = dev_params(p, L);
    void* copy = static_cast<char*>(const_cast<void*>(d_state)) + ((L.two && (t & 1)) ? L.copy : 0);
    const StateView st = view_of(p, L, copy);
    const int mode = L.two ? lbm::kModePull : ((t & 1) ? lbm::kModeAAOdd : lbm::kModeAAEven);
    double* partials = reinterpret_cast<double*>(w + L.off_partials);
    double* dout = reinterpret_cast<double*>(w + L.off_out);
    cudaGetLastError();
    LBM_DISPATCH(p->storage, launch_reduce, dp, st, p->lattice, p->flow != 0, mode, w + L.off_phi,
                 w + L.off_bits, partials, kRedBlocks, cs);
    reduce_final<<<1, 256, 0, cs>>>(partials, kRedBlocks, dout);
    s = cuda_check(nullptr, "static reduce launch");
    if (s != LBM_OK) return s;
    cudaError_t e = cudaMemcpyAsync(out, dout, LBM_NRED * sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, std::string("static reduce copy: ") + cudaGetErrorString(e));
    if (out[LBM_RED_NONFINITE] != 0.0)
        return fail(nullptr, LBM_ERR_UNSTABLE, "non-finite moments in the state (unstable run)");
    return LBM_OK;
}
