// Host orchestration of the PDE-EPDiff LDDMM hot path on one GPU.
//
// Engine<T> owns one device workspace and runs, on one CUDA stream:
//   * the spectral "program" planner that turns requests of the form
//       real_out = F^-1[ symbol . (sum_b c_b X_b) ]            (inverse)
//       spec_out = sum_b c_b B_b + sum_i symbol_i . F(real_i)  (forward)
//     into the three FFT passes (axis 0, axis 1, axis 2) with fan-out and
//     combination inside each pass; with the 2/3-rule projector P on, the
//     transforms of the shooting and of both Jacobi sweeps are band-limited:
//     the passes touch only the k2 planes and k1 columns of the band (every
//     source there is band-limited or read through P, every output is used
//     through P only; the adjoint state's out-of-band part never reaches its
//     band, since each operator of the transposed step maps out-of-band
//     input to out-of-band output);
//   * EPDiff shooting (Heun) with semi-Lagrangian map transport (Sec. 2.2,
//     Sec. 3 of the paper), storing every stage's v, Dv, m = Lv, Dm;
//   * the forward Jacobi (tangent) sweep and its exact transpose, the adjoint
//     Jacobi sweep (Sec. 3: incremental EPDiff and the reduced (incremental)
//     adjoint Jacobi equations with the Gauss-Newton drops);
//   * the reduced gradient, the Gauss-Newton Hessian-vector product, PCG with
//     preconditioner K and the Gauss-Newton-Krylov loop (Sec. 2.3, Sec. 3).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "fft_fast.cuh"
#include "fft_kernels.cuh"
#include "fused_stage.cuh"
#include "lddmm.h"
#include "pw_kernels.cuh"

namespace lddmm {

// NVTX range around a stage of the path (shoot, sweeps, gradient, Hv, GN and
// PCG iterations), visible to a profiler attached to the process; without
// one the push and pop cost a function-pointer test.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Kernel classes for the optional CUDA-event profiler.
enum KClass { KC_AX0 = 0, KC_AX1, KC_AX2, KC_ADSTAR, KC_TANPW, KC_ADJPW, KC_SL, KC_WARP, KC_RED, KC_SPEC, KC_MISC,
              KC_SCAN, KC_TANF, KC_ADJF, KC_COUNT };
static const char* const kclass_names[KC_COUNT] = {
    "fft_axis0_c2c", "fft_axis1_c2c", "fft_axis2_r2c_c2r", "adstar_pointwise", "tangent_pointwise",
    "adjoint_pointwise", "sl_map_step", "warp", "reduction", "spectral_combine", "misc_pointwise",
    "input_scan", "tangent_stage_fused", "adjoint_stage_fused"};

struct EngineBase {
    virtual ~EngineBase() {}
    virtual lddmm_status profile(int enable) = 0;
    virtual lddmm_status profile_read(int cls, double* ms, double* bytes, long long* launches) = 0;
    virtual lddmm_status shoot(const void* v0, const void* I0, void* m1, void* u1, double* kinetic) = 0;
    virtual lddmm_status gradient(const void* v0, const void* I0, const void* I1, void* grad, double* energy) = 0;
    virtual lddmm_status hessvec(const void* dv0, void* Hdv) = 0;
    virtual lddmm_status jacobi_forward(const void* dv0, void* eta1, void* xi1) = 0;
    virtual lddmm_status jacobi_adjoint(const void* beta, const void* bxi, void* out) = 0;
    virtual lddmm_status apply_metric(const void* in, void* out, int ncomp, int power) = 0;
    virtual lddmm_status jacobian_det(const void* u, void* J, double* minmax) = 0;
    virtual lddmm_status reg(const void* I0, const void* I1, void* v0, lddmm_report* rep) = 0;
    virtual lddmm_status synchronize() = 0;
    virtual lddmm_status shoot_vjp(const void* G, void* out) = 0;
    lddmm_status status = LDDMM_OK;
};

// ------------------------------------------------------------------ sizes
struct Dims {
    int n0, n1, n2, n2h;
    size_t N, NS, rows;
    double len[3], h[3], cell;
};

inline bool axis_ok(int n) {
    if (n < 2 || n > 512) return false;
    int m = n;
    for (int r : {2, 3, 5})
        while (m % r == 0) m /= r;
    return m == 1;
}

inline bool make_dims(const lddmm_grid* g, Dims* d) {
    if (!g) return false;
    for (int a = 0; a < 3; ++a)
        if (!axis_ok(g->n[a])) return false;
    d->n0 = g->n[0];
    d->n1 = g->n[1];
    d->n2 = g->n[2];
    d->n2h = d->n2 / 2 + 1;
    d->N = (size_t)d->n0 * d->n1 * d->n2;
    d->NS = (size_t)d->n0 * d->n1 * d->n2h;
    d->rows = (size_t)d->n0 * d->n1;
    d->cell = 1.0;
    for (int a = 0; a < 3; ++a) {
        d->len[a] = g->len[a] > 0 ? g->len[a] : 2.0 * M_PI;
        d->h[a] = d->len[a] / g->n[a];
        d->cell *= d->h[a];
    }
    return true;
}

constexpr int POOL = 64;   // partial spectra for the planner (a fused stage holds 57)
constexpr int RSCR = 42;   // real scratch fields
constexpr int NSLOT = 65;  // device double result slots
constexpr int SCAN_SLOT = 64;  // verdict of the non-finite input scan

// Pinned host result slots (NSLOT doubles per handle) from a process-wide
// free list, so that creating or destroying a handle neither allocates nor
// frees page-locked memory (either synchronises the whole device); they are
// allocated 64 handles' worth at a time and never freed.
inline std::mutex& pinned_mutex() {
    static std::mutex m;
    return m;
}
inline std::vector<double*>& pinned_free() {
    static std::vector<double*> v;
    return v;
}
inline double* pinned_slots_get() {
    std::lock_guard<std::mutex> g(pinned_mutex());
    std::vector<double*>& f = pinned_free();
    if (f.empty()) {
        constexpr int CHUNK = 64;
        double* b = nullptr;
        if (cudaMallocHost(&b, (size_t)CHUNK * NSLOT * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = CHUNK - 1; i >= 0; --i) f.push_back(b + (size_t)i * NSLOT);
    }
    double* p = f.back();
    f.pop_back();
    return p;
}
inline void pinned_slots_put(double* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(pinned_mutex());
    pinned_free().push_back(p);
}

// Workspace layout (element counts).  Shared by the allocator and by
// lddmm_workspace_bytes so admission control sees the true footprint.
struct Layout {
    size_t spec_fields, real_fields, bytes;
};
inline Layout layout_for(const Dims& d, const lddmm_params* p, size_t tsize) {
    Layout L;
    // pool + vhat(6) + v0hat(3) + v0full(3) + R1(3) + tan(12) + tb(6) + adj(12) + adja(6) + dhat(3) + tmp(3)
    L.spec_fields = POOL + 6 + 3 + 3 + 3 + 12 + 6 + 12 + 6 + 3 + 3;
    // vfin(6) + u(6) + scratch + m1(1) + gm1(3) + r(1) + Lv0(3) + PCG (x r z p q g vt: 21)
    // + FP32 copies of the last two stage-1 velocities for the map transport (6)
    const bool bf16 = p->state_dtype == LDDMM_BF16;
    const int cpe = p->checkpoint_every <= 1 ? p->nt : std::min(p->checkpoint_every, p->nt);
    const bool ckpt = cpe < p->nt;
    const int nseg = (p->nt + cpe - 1) / cpe;
    L.real_fields = 6 + 6 + RSCR + 1 + 3 + 1 + 3 + 21 + 6;
    // exact discrete gradient: every map u_k, every dE/dv_k, two dE/du buffers
    if (p->gradient_mode == LDDMM_GRAD_DISCRETE) L.real_fields += (size_t)6 * (p->nt + 1) + 6;
    if (ckpt) L.spec_fields += (size_t)3 * nseg;  // spectral v at the checkpoints
    size_t b = L.spec_fields * d.NS * 2 * tsize + L.real_fields * d.N * tsize;
    // stored time states: every stage, or one segment of checkpoint_every steps
    b += (size_t)2 * (ckpt ? cpe : p->nt) * 24 * d.N * (bf16 ? 2 : tsize);
    b += (size_t)(d.n0 + d.n1 + d.n2) * 2 * tsize * 2;  // twiddles
    b += (size_t)(d.n0 + d.n1 + d.n2h) * tsize * 2;      // symbol tables
    b += (RED_BLOCKS * 3 + NSLOT) * sizeof(double);
    b += 64 * 256;                                       // alignment slack
    L.bytes = b;
    return L;
}

// LDDMM_GENERIC_FFT=1 selects the generic (runtime-radix) passes for every
// axis; used to cross-check the register-blocked passes.
inline bool force_generic_fft() {
    const char* e = getenv("LDDMM_GENERIC_FFT");
    return e && e[0] == '1';
}
// LDDMM_SL_GATHER=1 makes the FP32 map steps use the global-gather kernel
// k_sl_step instead of the shared-memory staged one; used to cross-check the
// staged kernel, including its fallback for stencils that leave the box.
inline bool force_sl_gather() {
    const char* e = getenv("LDDMM_SL_GATHER");
    return e && e[0] == '1';
}
// LDDMM_UNFUSED=1 runs the Jacobi stages as separate axis-2 passes and
// pointwise kernels instead of the fused stage kernels (cross-check).
inline bool force_unfused() {
    const char* e = getenv("LDDMM_UNFUSED");
    return e && e[0] == '1';
}
// LDDMM_NO_GRAPH=1 launches the Hessian-vector product's kernels one by one
// instead of replaying its recorded CUDA graph (cross-check).
inline bool force_no_graph() {
    const char* e = getenv("LDDMM_NO_GRAPH");
    return e && e[0] == '1';
}
// LDDMM_FULL_BAND=1 transforms every spectral line even where the 2/3-rule
// band makes most of them zero; used to cross-check the band-limited passes.
inline bool force_full_band() {
    const char* e = getenv("LDDMM_FULL_BAND");
    return e && e[0] == '1';
}

inline std::vector<int> radix_plan(int n) {
    std::vector<int> r;
    int m = n;
    while (m % 4 == 0) {
        r.push_back(4);
        m /= 4;
    }
    while (m % 2 == 0) {
        r.push_back(2);
        m /= 2;
    }
    while (m % 3 == 0) {
        r.push_back(3);
        m /= 3;
    }
    while (m % 5 == 0) {
        r.push_back(5);
        m /= 5;
    }
    return r;
}

// The dynamic shared-memory limit of a kernel is process-wide: every site that
// raises it sets the device's opt-in maximum, so that a handle (or call) for a
// smaller grid never lowers the limit under a concurrent launch of a larger one.
inline int smem_optin_max() {
    int dev = 0, v = 48 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}
template <class K>
inline bool raise_smem_limit(K kernel, size_t need) {
    const int mx = smem_optin_max();
    if ((size_t)mx < need) return false;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess) return true;
    cudaGetLastError();  // a refusal must not stay pending: the caller falls back to another kernel
    return false;
}

// Ask for the smallest shared-memory carveout that holds `blocks` resident
// blocks of `bytes` dynamic shared memory each, so that the rest of the SM's
// unified L1/shared storage stays L1 (a hint: the driver rounds it up to a
// split it supports).
template <class K>
inline void prefer_l1(K kernel, size_t bytes, int blocks) {
    int dev = 0, per_sm = 0, resv = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        return;
    }
    const size_t need = (size_t)blocks * (bytes + (size_t)resv);
    const int pct = (int)std::min<size_t>(100, (need * 100 + (size_t)per_sm - 1) / (size_t)per_sm);
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
        cudaGetLastError();  // a hint only
}

// Grid of a persistent pass: `per_sm` resident blocks per SM, never more
// blocks than work items.
inline int persistent_grid(int items, int per_sm = 3) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return std::max(1, std::min(items, per_sm * sms));
}

// Launch of the register-blocked passes for the compiled line lengths.
template <class T> struct FastPass {
    // the persistent axis-2 kernel's shared-memory limit is raised (per N)
    template <int N> static bool& a2p_ready() {
        static bool v = false;
        return v;
    }
    // The persistent axis-2 kernel takes full tiles of r2 rows, one input per
    // inverse job, and 16-byte aligned inputs (its copies are 16-byte
    // cp.async of whole rows or plane segments).
    static bool axis2p_fits(const PassParams<T>& pp, int nj, size_t rows, int r2) {
        if (rows % (size_t)r2 != 0 || (rows / r2) * (size_t)nj >= (1u << 24)) return false;
        for (int j = 0; j < nj; ++j) {
            const PassJobT<T>& jb = pp.jobs[j];
            if (pp.sign > 0 && jb.nin != 1) return false;
            for (int i = 0; i < jb.nin; ++i)
                if ((uintptr_t)jb.in[i] % 16 != 0) return false;
        }
        return true;
    }
    template <int N>
    static bool go(int axis, int sign, PassParams<T>& pp, int nj, size_t rows, int n0, int n1, int n2h,
                   cudaStream_t st, bool set_attr) {
        (void)sign;
        constexpr int TL = FAST_THREADS / (N / FastPlan<N>::E);
        if (axis == 2) {
            const size_t sm = fast_axis2_smem<T, N>();
            constexpr bool PERS = sizeof(T) == 4 && FastPlan<N>::E <= 12;
            if (set_attr) {
                if constexpr (PERS) a2p_ready<N>() = raise_smem_limit(k_fast_axis2p<T, N>, fast_axis2p_smem<T, N>());
                return raise_smem_limit(k_fast_axis2<T, N>, sm);
            }
            if constexpr (PERS) {
                if (a2p_ready<N>() && axis2p_fits(pp, nj, rows, 2 * TL)) {
                    const int ntiles = (int)(rows / (2 * TL));
                    pp.fd_tiles = FastDiv((unsigned)ntiles);
                    k_fast_axis2p<T, N><<<persistent_grid(ntiles * nj, A2P_BLOCKS), FAST_THREADS, fast_axis2p_smem<T, N>(),
                                          st>>>(pp, ntiles);
                    return true;
                }
            }
            const int gx = (int)((rows + 2 * TL - 1) / (2 * TL));
            k_fast_axis2<T, N><<<dim3(gx, nj), FAST_THREADS, sm, st>>>(pp);
        } else if (axis == 1) {
            const size_t sm = fast_c2c_smem<T, N>(1);
            if (set_attr) {
                if (!raise_smem_limit(k_fast_c2c<T, N, 1>, sm)) return false;
                prefer_l1(k_fast_c2c<T, N, 1>, sm, FastOccC2C<T, N>::value);
                return true;
            }
            (void)n2h;
            const int ntiles = (int)(((size_t)pp.nb2 * n0 + TL - 1) / TL);
            pp.fd_tiles = FastDiv((unsigned)ntiles);
            pp.fd_n0 = FastDiv((unsigned)n0);
            k_fast_c2c<T, N, 1><<<persistent_grid(ntiles * nj), FAST_THREADS, sm, st>>>(pp, ntiles);
        } else {
            const size_t sm = fast_c2c_smem<T, N>(0);
            if (set_attr) {
                if (!raise_smem_limit(k_fast_c2c<T, N, 0>, sm)) return false;
                prefer_l1(k_fast_c2c<T, N, 0>, sm, FastOccC2C<T, N>::value);
                return true;
            }
            const int tpk = (pp.c1 + TL - 1) / TL + (n1 - pp.s1 + TL - 1) / TL;
            const int ntiles = pp.nb2 * tpk;
            pp.fd_tiles = FastDiv((unsigned)ntiles);
            pp.fd_tpk = FastDiv((unsigned)tpk);
            k_fast_c2c<T, N, 0><<<persistent_grid(ntiles * nj), FAST_THREADS, sm, st>>>(pp, ntiles);
        }
        return true;
    }
    // n: the line length of this axis.  Returns false when no plan exists.
    static bool launch(int n, int axis, int sign, PassParams<T>& pp, int nj, size_t rows, int n0, int n1, int n2h,
                       cudaStream_t st, bool set_attr = false) {
        switch (n) {
            case 32: return go<32>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            case 64: return go<64>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            case 128: return go<128>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            case 256: return go<256>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            case 96: return go<96>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            case 160: return go<160>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            case 192: return go<192>(axis, sign, pp, nj, rows, n0, n1, n2h, st, set_attr);
            default: return false;
        }
    }
    static bool has(int n) { return n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 192 || n == 256; }
};

// Launch of the fused Jacobi stage kernels (FP32, n2 with an E = 8 plan).
struct FusedPass {
    static bool has(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }
    static int tile_rows(int n) { return FAST_THREADS / (n / 8); }
    static int band_planes(int n) { return (n - 1) / 3 + 1; }  // FusedGeom<n>::NB2
    template <int N, class SS, int KIND> static bool go(const FusedArgs& a, cudaStream_t st, bool set_attr) {
        if (set_attr) {
            if (!raise_smem_limit(k_fused_stage<SS, N, KIND>, FusedGeom<N>::smem(KIND))) return false;
            prefer_l1(k_fused_stage<SS, N, KIND>, FusedGeom<N>::smem(KIND), FUSED_BLOCKS);
            return true;
        }
        if (a.nb2 != FusedGeom<N>::NB2) return false;
        const size_t sm = FusedGeom<N>::smem(KIND);
        k_fused_stage<SS, N, KIND><<<persistent_grid(a.ntiles, FUSED_BLOCKS), FAST_THREADS, sm, st>>>(a);
        return true;
    }
    template <class SS, int KIND>
    static bool launch(int n, const FusedArgs& a, cudaStream_t st, bool set_attr = false) {
        switch (n) {
            case 32: return go<32, SS, KIND>(a, st, set_attr);
            case 64: return go<64, SS, KIND>(a, st, set_attr);
            case 128: return go<128, SS, KIND>(a, st, set_attr);
            case 256: return go<256, SS, KIND>(a, st, set_attr);
            default: return false;
        }
    }
    static bool prepare(int n) {
        return launch<float, 0>(n, FusedArgs{}, 0, true) && launch<float, 1>(n, FusedArgs{}, 0, true) &&
               launch<__nv_bfloat16, 0>(n, FusedArgs{}, 0, true) && launch<__nv_bfloat16, 1>(n, FusedArgs{}, 0, true);
    }
};

#define LD_CK(call)                                           \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return fail(LDDMM_ERR_CUDA);   \
    } while (0)

template <class T>
class Engine : public EngineBase {
   public:
    using C = cpx<T>;

    struct SpecLin {
        const C* p[MAXI];
        double c[MAXI];
        int n;
    };
    struct InvReq {
        int src;
        SymD sym;
        T* out;
    };
    struct FwdTerm {
        const T* in;
        SymD sym;
    };
    struct FwdOut {
        C* out;
        std::vector<FwdTerm> terms;
        std::vector<std::pair<const C*, double>> bases;
    };

    Dims d;
    lddmm_params prm;
    cudaStream_t st;
    unsigned char* base_ = nullptr;
    size_t off_ = 0, cap_ = 0;

    // device buffers
    C* pool[POOL];
    C *vhat[2], *v0hat, *v0full, *R1, *tan_[2], *tb, *adj[2], *adja, *dhat, *tmp;
    void* states;  // 2 nt stages (or 2 checkpoint_every stages) x 24 fields, T or bfloat16
    bool bf16 = false;
    // checkpointing: v-hat kept every cpe steps, states of one segment resident
    int cpe = 1, nseg = 1, seg_res = -1;
    bool ckpt = false;
    C* cps = nullptr;
    T *vfin, *ubuf[2], *rs, *m1, *gm1, *rbuf, *lv0, *vss[2] = {nullptr, nullptr};
    // exact discrete gradient: maps u_k (k = 0..nt), dE/dv_k, dE/du ping-pong
    T *ustore = nullptr, *vbar = nullptr, *ubar[2] = {nullptr, nullptr};
    bool exact_grad = false;
    T *px, *pr, *pz, *pp, *pq, *pg, *pvt;
    double *partial, *dres, *hres = nullptr;
    cudaEvent_t scan_ev = nullptr;
    bool scan_pending = false;
    FFTAxis ax[3];
    SpecTabs<T> tabs;
    int TLc[2], Pc[2], TL2, P2, Ph2;
    bool fast[3] = {false, false, false};
    // band-limited transforms (all three passes register-blocked, dealiasing on)
    bool band_ok = false;
    bool sl_staged = false;  // FP32 map steps use k_sl_step_staged
    bool fused = false;      // FP32 Jacobi stages use k_fused_stage
    int bnb2 = 0, bc1 = 0, bs1 = 0;
    size_t smem_c[2], smem2;
    int pool_top = 0;
    bool lin_valid = false;

    // ---- optional kernel profiler: CUDA events around every launch
    struct PendingEv {
        int i0, i1, cls;
        double bytes;
    };
    bool prof_on = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    std::vector<PendingEv> pend;
    double acc_ms[KC_COUNT] = {}, acc_bytes[KC_COUNT] = {};
    long long acc_n[KC_COUNT] = {};

    void prof_flush() {
        if (pend.empty()) return;
        cudaStreamSynchronize(st);
        for (const PendingEv& q : pend) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[q.i0], ev[q.i1]);
            acc_ms[q.cls] += ms;
            acc_bytes[q.cls] += q.bytes;
            acc_n[q.cls] += 1;
        }
        pend.clear();
        ev_used = 0;
    }
    struct PScope {
        Engine* e;
        int cls, i0;
        double bytes;
        PScope(Engine* e_, int c, double b) : e(e_), cls(c), i0(-1), bytes(b) {
            if (!e->prof_on) return;
            if (e->ev_used + 2 > (int)e->ev.size()) e->prof_flush();
            i0 = e->ev_used++;
            cudaEventRecord(e->ev[i0], e->st);
        }
        ~PScope() {
            if (i0 < 0) return;
            const int i1 = e->ev_used++;
            cudaEventRecord(e->ev[i1], e->st);
            e->pend.push_back({i0, i1, cls, bytes});
        }
    };
    lddmm_status profile(int enable) override {
        if (enable) {
            if (ev.empty()) {
                ev.resize(8192);
                for (auto& x : ev)
                    if (cudaEventCreate(&x) != cudaSuccess) return fail(LDDMM_ERR_CUDA);
            }
            prof_flush();
            for (int c = 0; c < KC_COUNT; ++c) acc_ms[c] = acc_bytes[c] = 0, acc_n[c] = 0;
            prof_on = true;
        } else {
            prof_flush();
            prof_on = false;
        }
        return status;
    }
    lddmm_status profile_read(int cls, double* ms, double* bytes, long long* launches) override {
        if (cls < 0 || cls >= KC_COUNT) return LDDMM_ERR_ARG;
        prof_flush();
        if (ms) *ms = acc_ms[cls];
        if (bytes) *bytes = acc_bytes[cls];
        if (launches) *launches = acc_n[cls];
        return status;
    }
    // Compulsory bytes of a pass: the spectral entries of the band it
    // transforms (fp: planes, fc: k1 columns) and the real rows.
    double pass_bytes(int axis, int sign, const PassParams<T>& q) const {
        double b = 0;
        const double sc = (double)d.NS * sizeof(C), sr = (double)d.N * sizeof(T);
        const double fp = (double)q.nb2 / d.n2h, fc = (double)(q.c1 + d.n1 - q.s1) / d.n1;
        for (int j = 0; j < q.njobs; ++j) {
            const PassJobT<T>& jb = q.jobs[j];
            if (axis == 0) b += (jb.nin + jb.nb + jb.nout) * sc * fp * fc;
            else if (axis == 1) b += (sign > 0 ? jb.nin * fc + jb.nout : jb.nin + jb.nout * fc) * sc * fp;
            else if (sign > 0) b += jb.nin * sc * fp + jb.nout * sr;
            else b += jb.nin * sr + sc * fp;
        }
        return b;
    }

    Engine(const Dims& dd, const lddmm_params& p, cudaStream_t s) : d(dd), prm(p), st(s) {}

    ~Engine() override {
        if (hvg.exec) cudaGraphExecDestroy(hvg.exec);
        for (auto& x : ev) cudaEventDestroy(x);
        if (scan_ev) cudaEventDestroy(scan_ev);
        // stream-ordered: the workspace returns to the pool after the
        // stream's queued work, with no device-wide synchronisation
        if (base_) cudaFreeAsync(base_, st);
        pinned_slots_put(hres);
    }

    lddmm_status fail(lddmm_status s) {
        if (status == LDDMM_OK) status = s;
        return status;
    }

    template <class U>
    U* carve(size_t count) {
        size_t o = (off_ + 255) & ~(size_t)255;
        U* p = (U*)(base_ + o);
        off_ = o + count * sizeof(U);
        return p;
    }

    lddmm_status init() {
        Layout L = layout_for(d, &prm, sizeof(T));
        cap_ = L.bytes;
        // Set-up stays on the handle's stream (stream-ordered allocation,
        // asynchronous fills and copies, one stream synchronisation), so that
        // creating a handle does not wait for other handles' queued work.
        if (cudaMallocAsync((void**)&base_, cap_, st) != cudaSuccess) {
            base_ = nullptr;
            cudaGetLastError();
            return fail(LDDMM_ERR_OOM);
        }
        hres = pinned_slots_get();
        if (!hres) return fail(LDDMM_ERR_OOM);
        if (cudaEventCreateWithFlags(&scan_ev, cudaEventDisableTiming) != cudaSuccess) {
            scan_ev = nullptr;
            return fail(LDDMM_ERR_CUDA);
        }
        for (int i = 0; i < POOL; ++i) pool[i] = carve<C>(d.NS);
        for (int i = 0; i < 2; ++i) vhat[i] = carve<C>(3 * d.NS);
        v0hat = carve<C>(3 * d.NS);
        v0full = carve<C>(3 * d.NS);
        R1 = carve<C>(3 * d.NS);
        for (int i = 0; i < 2; ++i) tan_[i] = carve<C>(6 * d.NS);
        tb = carve<C>(6 * d.NS);
        for (int i = 0; i < 2; ++i) adj[i] = carve<C>(6 * d.NS);
        adja = carve<C>(6 * d.NS);
        dhat = carve<C>(3 * d.NS);
        tmp = carve<C>(3 * d.NS);
        bf16 = prm.state_dtype == LDDMM_BF16;
        cpe = prm.checkpoint_every <= 1 ? prm.nt : std::min(prm.checkpoint_every, prm.nt);
        ckpt = cpe < prm.nt;
        nseg = (prm.nt + cpe - 1) / cpe;
        const size_t nstate = (size_t)2 * (ckpt ? cpe : prm.nt) * 24 * d.N;
        if (bf16) states = carve<__nv_bfloat16>(nstate);
        else states = carve<T>(nstate);
        for (int i = 0; i < 2; ++i) vss[i] = carve<T>(3 * d.N);
        if (ckpt) cps = carve<C>((size_t)3 * nseg * d.NS);
        vfin = carve<T>(6 * d.N);
        for (int i = 0; i < 2; ++i) ubuf[i] = carve<T>(3 * d.N);
        exact_grad = prm.gradient_mode == LDDMM_GRAD_DISCRETE;
        if (exact_grad) {
            ustore = carve<T>((size_t)3 * (prm.nt + 1) * d.N);
            vbar = carve<T>((size_t)3 * (prm.nt + 1) * d.N);
            for (int i = 0; i < 2; ++i) ubar[i] = carve<T>(3 * d.N);
        }
        rs = carve<T>((size_t)RSCR * d.N);
        m1 = carve<T>(d.N);
        gm1 = carve<T>(3 * d.N);
        rbuf = carve<T>(d.N);
        lv0 = carve<T>(3 * d.N);
        px = carve<T>(3 * d.N);
        pr = carve<T>(3 * d.N);
        pz = carve<T>(3 * d.N);
        pp = carve<T>(3 * d.N);
        pq = carve<T>(3 * d.N);
        pg = carve<T>(3 * d.N);
        pvt = carve<T>(3 * d.N);
        partial = carve<double>(RED_BLOCKS * 3);
        dres = carve<double>(NSLOT);
        // LDDMM_POISON_WORKSPACE=1 fills the buffers with NaN bytes instead of
        // zeros, so that a test sees any read of an entry never written.
        const char* poison = getenv("LDDMM_POISON_WORKSPACE");
        LD_CK(cudaMemsetAsync(base_, poison && poison[0] == '1' ? 0xFF : 0, off_, st));
        LD_CK(cudaMemsetAsync(dres + SCAN_SLOT, 0, sizeof(double), st));
        // twiddles and symbol tables
        const int ns[3] = {d.n0, d.n1, d.n2};
        for (int a = 0; a < 3; ++a) {
            const int n = ns[a];
            std::vector<int> rp = radix_plan(n);
            ax[a].n = n;
            ax[a].nst = (int)rp.size();
            for (int i = 0; i < (int)rp.size(); ++i) ax[a].rad[i] = rp[i];
            std::vector<C> tw(n);
            for (int t = 0; t < n; ++t) {
                long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)n;
                tw[t].x = (T)cosl(ang);
                tw[t].y = (T)sinl(ang);
            }
            C* dtw = carve<C>(n);
            // pageable source: the call returns once the data is staged
            LD_CK(cudaMemcpyAsync(dtw, tw.data(), n * sizeof(C), cudaMemcpyHostToDevice, st));
            ax[a].tw = dtw;
        }
        const int nk[3] = {d.n0, d.n1, d.n2h};
        for (int a = 0; a < 3; ++a) {
            std::vector<T> dk(nk[a]), ks(nk[a]);
            const int n = ns[a];
            for (int k = 0; k < nk[a]; ++k) {
                int sk = (a < 2 && k >= (n + 1) / 2) ? k - n : k;
                double kap = 2.0 * M_PI / d.len[a] * sk;
                ks[k] = (T)(kap * kap);
                bool nyq = (n % 2 == 0) && (k == n / 2);
                dk[k] = nyq ? (T)0 : (T)kap;
            }
            T* ddk = carve<T>(nk[a]);
            T* dks = carve<T>(nk[a]);
            LD_CK(cudaMemcpyAsync(ddk, dk.data(), nk[a] * sizeof(T), cudaMemcpyHostToDevice, st));
            LD_CK(cudaMemcpyAsync(dks, ks.data(), nk[a] * sizeof(T), cudaMemcpyHostToDevice, st));
            tabs.dk[a] = ddk;
            tabs.ksq[a] = dks;
        }
        tabs.alpha = (T)prm.alpha;
        tabs.s = prm.s;
        for (int a = 0; a < 3; ++a) {
            tabs.n[a] = ns[a];
            tabs.kcut[a] = prm.dealias ? (ns[a] - 1) / 3 : ns[a];
        }
        if (off_ > cap_) return fail(LDDMM_ERR_OOM);
        // tile geometry
        const size_t budget = 150 * 1024;
        for (int a = 0; a < 2; ++a) {
            const int n = ns[a];
            Pc[a] = (n % 2 == 0) ? n + 1 : n;
            TLc[a] = 16;
            while (TLc[a] > 1 && (size_t)3 * TLc[a] * Pc[a] * sizeof(C) > budget) TLc[a] /= 2;
            smem_c[a] = (size_t)3 * TLc[a] * Pc[a] * sizeof(C);
        }
        P2 = (d.n2 % 2 == 0) ? d.n2 + 1 : d.n2;
        Ph2 = (d.n2h % 2 == 0) ? d.n2h + 1 : d.n2h;
        TL2 = 16;
        while (TL2 > 1 && ((size_t)2 * TL2 * Ph2 + 2 * TL2 * P2) * sizeof(C) > budget) TL2 /= 2;
        smem2 = ((size_t)2 * TL2 * Ph2 + 2 * TL2 * P2) * sizeof(C);
        if (!raise_smem_limit(k_pass_c2c<T, 0>, smem_c[0]) || !raise_smem_limit(k_pass_c2c<T, 1>, smem_c[1]) ||
            !raise_smem_limit(k_pass_axis2<T>, smem2))
            return fail(LDDMM_ERR_CUDA);
        for (int a = 0; a < 3; ++a) {
            PassParams<T> dummy;
            // 16-byte copies of axis-0 tile rows need an even n1 in FP32
            const bool aligned = a != 0 || sizeof(T) == 8 || ns[1] % 2 == 0;
            fast[a] = FastPass<T>::has(ns[a]) && aligned && !force_generic_fft() &&
                      FastPass<T>::launch(ns[a], a, 0, dummy, 0, 0, 0, 0, 0, st, true);
        }
        // the 2/3-rule band: k2 <= kcut2; k1 columns rounded outwards to even
        // indices (16-byte copies of FP32 pairs)
        bnb2 = std::min(tabs.kcut[2] + 1, d.n2h);
        bc1 = (tabs.kcut[1] + 2) & ~1;
        bs1 = (d.n1 - tabs.kcut[1]) & ~1;
        if (bc1 >= bs1) bc1 = bs1 = d.n1;
        if constexpr (sizeof(T) == 4)
            sl_staged = !force_sl_gather() && raise_smem_limit(k_sl_step_staged<true>, SLBox<true>::SMEM) &&
                        raise_smem_limit(k_sl_step_staged<false>, SLBox<false>::SMEM);
        band_ok = prm.dealias && fast[0] && fast[1] && fast[2] && !force_full_band() &&
                  (bnb2 < d.n2h || bc1 < bs1);
        if constexpr (sizeof(T) == 4)
            fused = band_ok && !force_unfused() && FusedPass::has(d.n2) && bnb2 == FusedPass::band_planes(d.n2) &&
                    d.rows % (size_t)FusedPass::tile_rows(d.n2) == 0 && FusedPass::prepare(d.n2);
        LD_CK(cudaStreamSynchronize(st));
        return LDDMM_OK;
    }

    // ------------------------------------------------------------ helpers
    C* palloc() {
        if (pool_top >= POOL) {
            fail(LDDMM_ERR_DEVICE_CHECK);
            return pool[POOL - 1];
        }
        return pool[pool_top++];
    }
    int pw_grid(size_t n) const { return (int)std::min<size_t>((n + PW_THREADS - 1) / PW_THREADS, 152 * 16); }
    // element offset of global stage s in the state store (the resident
    // segment's local index under checkpointing)
    size_t sofs(int s) const {
        const int l = ckpt ? s - 2 * cpe * seg_res : s;
        if (l < 0 || l >= 2 * (ckpt ? cpe : prm.nt)) {
            const_cast<Engine*>(this)->fail(LDDMM_ERR_DEVICE_CHECK);
            return 0;
        }
        return (size_t)l * 24 * d.N;
    }
    T* state(int s) const { return (T*)states + sofs(s); }
    // the map u_k: every step kept for the exact discrete gradient, else two
    // ping-pong buffers
    T* ubuf_at(int k) const { return exact_grad ? ustore + (size_t)3 * k * d.N : ubuf[k % 2]; }
    __nv_bfloat16* state_bf(int s) const { return (__nv_bfloat16*)states + sofs(s); }
    double state_elem() const { return bf16 ? 2.0 : (double)sizeof(T); }
    double dt() const { return 1.0 / prm.nt; }

    void launch(int axis, int sign, std::vector<PassJob>& jobs, bool band) {
        for (size_t j0 = 0; j0 < jobs.size(); j0 += MAXJOBS) {
            const int nj = (int)std::min<size_t>(MAXJOBS, jobs.size() - j0);
            PassParams<T> pp_;
            pp_.ax = ax[axis];
            pp_.n0 = d.n0;
            pp_.n1 = d.n1;
            pp_.n2 = d.n2;
            pp_.n2h = d.n2h;
            pp_.sign = sign;
            full_band(pp_);
            if (band) {
                pp_.nb2 = bnb2;
                pp_.c1 = bc1;
                pp_.s1 = bs1;
            }
            pp_.tabs = tabs;
            pp_.njobs = nj;
            for (int j = 0; j < nj; ++j) pp_.jobs[j] = to_jobt<T>(jobs[j0 + j]);
            if (fast[axis]) {
                const int n = axis == 0 ? d.n0 : (axis == 1 ? d.n1 : d.n2);
                PScope ps_(this, axis == 0 ? KC_AX0 : (axis == 1 ? KC_AX1 : KC_AX2), pass_bytes(axis, sign, pp_));
                FastPass<T>::launch(n, axis, sign, pp_, nj, d.rows, d.n0, d.n1, d.n2h, st);
            } else if (axis == 2) {
                pp_.TL = TL2;
                pp_.P = P2;
                pp_.Ph = Ph2;
                const int gx = (int)((d.rows + 2 * TL2 - 1) / (2 * TL2));
                {
                    PScope ps_(this, KC_AX2, pass_bytes(2, sign, pp_));
                    k_pass_axis2<T><<<dim3(gx, nj), FFT_THREADS, smem2, st>>>(pp_);
                }
            } else if (axis == 1) {
                pp_.TL = TLc[1];
                pp_.P = Pc[1];
                pp_.Ph = 0;
                const int gx = (int)(((size_t)d.n2h * d.n0 + TLc[1] - 1) / TLc[1]);
                {
                    PScope ps_(this, KC_AX1, pass_bytes(1, sign, pp_));
                    k_pass_c2c<T, 1><<<dim3(gx, nj), FFT_THREADS, smem_c[1], st>>>(pp_);
                }
            } else {
                pp_.TL = TLc[0];
                pp_.P = Pc[0];
                pp_.Ph = 0;
                const int gx = d.n2h * ((d.n1 + TLc[0] - 1) / TLc[0]);
                {
                    PScope ps_(this, KC_AX0, pass_bytes(0, sign, pp_));
                    k_pass_c2c<T, 0><<<dim3(gx, nj), FFT_THREADS, smem_c[0], st>>>(pp_);
                }
            }
        }
    }

    static PassJob blank() {
        PassJob j;
        memset(&j, 0, sizeof(j));
        return j;
    }
    static SymD sym(double s, int l, int dv, int mask = 0) {
        SymD y;
        y.scale = s;
        y.lpow = l;
        y.deriv = dv;
        y.mask = mask;
        return y;
    }
    // out (3 spectral comps) = P in
    void mask_copy(const C* in, C* out) {
        for (int c = 0; c < 3; ++c) {
            SpecComb<T> sc;
            sc.nin = 1;
            sc.in[0] = in + c * d.NS;
            sc.sym[0] = to_symt<T>(sym(1.0, 0, -1, 1));
            {
                PScope ps_(this, KC_SPEC, 2.0 * d.NS * sizeof(C));
                k_spec_comb<T><<<spec_comb_blocks(d.n0, d.n2h), spec_comb_threads(d.n1), 0, st>>>(sc, tabs, d.n0, d.n1,
                                                                                               d.n2h, out + c * d.NS);
            }
        }
    }
    // slot = <L v0, v0> (regulariser of the energy), from F(v0) in v0full
    void reg_async(const T* v0, int slot) {
        std::vector<SpecLin> srcs;
        std::vector<InvReq> reqs;
        for (int c = 0; c < 3; ++c) {
            SpecLin s;
            s.n = 1;
            s.p[0] = v0full + c * d.NS;
            s.c[0] = 1.0;
            srcs.push_back(s);
            reqs.push_back({c, sym(1.0, 1, -1), lv0 + c * d.N});
        }
        inverse(srcs, reqs);
        dot_async(lv0, v0, 3 * d.N, slot, d.cell);
    }

    // The axis-2 inputs of an inverse transform: request r reads spectrum
    // k1[r1[r]] (after the axis-0 and axis-1 passes), with i kappa_2 applied
    // when d2[r].
    struct InvHead {
        std::vector<C*> k1;
        std::vector<int> r1;
        std::vector<char> d2;
        bool bd;
    };

    // real_out = F^-1[ sym . lincomb(src) ]
    // band: every source is band-limited or every request is masked, so the
    // transform may read the band only (the requests then all carry P).
    void inverse(const std::vector<SpecLin>& srcs, const std::vector<InvReq>& reqs, bool band = false) {
        const InvHead ih = inverse_head(srcs, reqs, band);
        std::vector<PassJob> jobs;
        for (size_t i1 = 0; i1 < ih.k1.size(); ++i1) {
            PassJob j = blank();
            auto setin = [&]() {
                j.nin = 1;
                j.in[0] = ih.k1[i1];
                j.isym[0] = sym(1.0, 0, -1);
            };
            setin();
            for (size_t r = 0; r < reqs.size(); ++r) {
                if (ih.r1[r] != (int)i1) continue;
                if (j.nout == MAXO) {
                    jobs.push_back(j);
                    j = blank();
                    setin();
                }
                j.out[j.nout] = reqs[r].out;
                j.osym[j.nout] = sym(1.0, 0, ih.d2[r] ? 2 : -1);
                j.nout++;
            }
            if (j.nout) jobs.push_back(j);
        }
        launch(2, +1, jobs, ih.bd);
    }

    // The axis-0 and axis-1 passes of inverse(), with the fan-out shared as a
    // tree; the pool's partial spectra hold the results.
    InvHead inverse_head(const std::vector<SpecLin>& srcs, const std::vector<InvReq>& reqs_in, bool band) {
        const bool bd = band && band_ok;
        std::vector<InvReq> reqs = reqs_in;
        if (bd)
            for (InvReq& q : reqs) q.sym.mask = 1;
        pool_top = 0;
        const double invN = 1.0 / (double)d.N;
        struct K0 {
            int src, lpow;
            double scale;
            bool d0;
            int mask;
            C* buf;
        };
        struct K1 {
            int k0;
            bool d1;
            C* buf;
        };
        std::vector<K0> k0s;
        std::vector<K1> k1s;
        std::vector<int> r0(reqs.size()), r1(reqs.size());
        for (size_t r = 0; r < reqs.size(); ++r) {
            const InvReq& q = reqs[r];
            const bool d0 = q.sym.deriv == 0;
            int f = -1;
            for (size_t i = 0; i < k0s.size(); ++i)
                if (k0s[i].src == q.src && k0s[i].lpow == q.sym.lpow && k0s[i].scale == q.sym.scale &&
                    k0s[i].d0 == d0 && k0s[i].mask == q.sym.mask)
                    f = (int)i;
            if (f < 0) {
                k0s.push_back({q.src, q.sym.lpow, q.sym.scale, d0, q.sym.mask, palloc()});
                f = (int)k0s.size() - 1;
            }
            r0[r] = f;
        }
        for (size_t r = 0; r < reqs.size(); ++r) {
            const bool d1 = reqs[r].sym.deriv == 1;
            int f = -1;
            for (size_t i = 0; i < k1s.size(); ++i)
                if (k1s[i].k0 == r0[r] && k1s[i].d1 == d1) f = (int)i;
            if (f < 0) {
                k1s.push_back({r0[r], d1, palloc()});
                f = (int)k1s.size() - 1;
            }
            r1[r] = f;
        }
        // axis 0
        std::vector<PassJob> jobs;
        for (size_t s = 0; s < srcs.size(); ++s) {
            PassJob j = blank();
            auto flush = [&]() {
                if (j.nout) jobs.push_back(j);
                PassJob b = blank();
                j = b;
            };
            auto setin = [&]() {
                j.nin = srcs[s].n;
                for (int b = 0; b < srcs[s].n; ++b) {
                    j.in[b] = srcs[s].p[b];
                    j.isym[b] = sym(srcs[s].c[b], 0, -1);
                }
            };
            setin();
            for (size_t i = 0; i < k0s.size(); ++i) {
                if (k0s[i].src != (int)s) continue;
                if (j.nout == MAXO) {
                    flush();
                    setin();
                }
                j.out[j.nout] = k0s[i].buf;
                j.osym[j.nout] = sym(k0s[i].scale * invN, k0s[i].lpow, k0s[i].d0 ? 0 : -1, k0s[i].mask);
                j.nout++;
            }
            flush();
        }
        launch(0, +1, jobs, bd);
        // axis 1
        jobs.clear();
        for (size_t i0 = 0; i0 < k0s.size(); ++i0) {
            PassJob j = blank();
            j.nin = 1;
            j.in[0] = k0s[i0].buf;
            j.isym[0] = sym(1.0, 0, -1);
            for (size_t i = 0; i < k1s.size(); ++i) {
                if (k1s[i].k0 != (int)i0) continue;
                j.out[j.nout] = k1s[i].buf;
                j.osym[j.nout] = sym(1.0, 0, k1s[i].d1 ? 1 : -1);
                j.nout++;
            }
            if (j.nout) jobs.push_back(j);
        }
        launch(1, +1, jobs, bd);
        InvHead ih;
        ih.bd = bd;
        for (const K1& k : k1s) ih.k1.push_back(k.buf);
        ih.r1 = r1;
        for (const InvReq& q : reqs) ih.d2.push_back(q.sym.deriv == 2);
        return ih;
    }

    // spec_out = sum bases + sum_i sym_i . F(real_i)
    // band: only the band of the output is ever used (it is masked, or every
    // consumer applies P), so the transform writes the band only, with P.
    // An axis-2 output of a forward transform: the partial spectrum of the
    // terms of output o with the same (lpow, scale, mask) whose derivative is
    // along axis 0 (cls 0), axis 1 (cls 1), or axis 2 / none (cls 2).
    struct G {
        int o, lpow;
        double scale;
        int cls, mask;
        C* buf;
        int nin;
    };
    void forward(const std::vector<FwdOut>& outs_in, bool band = false) {
        const bool bd = band && band_ok;
        std::vector<FwdOut> outs = outs_in;
        if (bd)
            for (FwdOut& o : outs)
                for (FwdTerm& t : o.terms) t.sym.mask = 1;
        pool_top = 0;
        // axis 2
        std::vector<G> g2;
        std::vector<PassJob> j2;
        for (size_t o = 0; o < outs.size(); ++o) {
            for (const FwdTerm& t : outs[o].terms) {
                const int cls = t.sym.deriv == 0 ? 0 : (t.sym.deriv == 1 ? 1 : 2);
                int f = -1;
                for (size_t i = 0; i < g2.size(); ++i)
                    if (g2[i].o == (int)o && g2[i].lpow == t.sym.lpow && g2[i].scale == t.sym.scale &&
                        g2[i].cls == cls && g2[i].mask == t.sym.mask && g2[i].nin < MAXI)
                        f = (int)i;
                if (f < 0) {
                    g2.push_back({(int)o, t.sym.lpow, t.sym.scale, cls, t.sym.mask, palloc(), 0});
                    PassJob j = blank();
                    j.nout = 1;
                    j.out[0] = g2.back().buf;
                    j2.push_back(j);
                    f = (int)g2.size() - 1;
                }
                PassJob& j = j2[f];
                j.in[j.nin] = t.in;
                j.isym[j.nin] = sym(1.0, 0, t.sym.deriv == 2 ? 2 : -1);
                j.nin++;
                g2[f].nin++;
            }
        }
        launch(2, -1, j2, bd);
        forward_tail(outs, g2, bd);
    }

    // The axis-1 and axis-0 passes of forward(), from its axis-2 outputs g2.
    void forward_tail(const std::vector<FwdOut>& outs, const std::vector<G>& g2, bool bd) {
        // axis 1
        std::vector<G> g1;
        std::vector<PassJob> j1;
        for (const G& a : g2) {
            const int cls0 = a.cls == 0 ? 0 : 1;
            int f = -1;
            for (size_t i = 0; i < g1.size(); ++i)
                if (g1[i].o == a.o && g1[i].lpow == a.lpow && g1[i].scale == a.scale && g1[i].cls == cls0 &&
                    g1[i].mask == a.mask && g1[i].nin < MAXI)
                    f = (int)i;
            if (f < 0) {
                g1.push_back({a.o, a.lpow, a.scale, cls0, a.mask, palloc(), 0});
                PassJob j = blank();
                j.nout = 1;
                j.out[0] = g1.back().buf;
                j1.push_back(j);
                f = (int)g1.size() - 1;
            }
            PassJob& j = j1[f];
            j.in[j.nin] = a.buf;
            j.isym[j.nin] = sym(1.0, 0, a.cls == 1 ? 1 : -1);
            j.nin++;
            g1[f].nin++;
        }
        launch(1, -1, j1, bd);
        // axis 0
        std::vector<PassJob> j0;
        for (size_t o = 0; o < outs.size(); ++o) {
            PassJob j = blank();
            j.nout = 1;
            j.out[0] = outs[o].out;
            for (const G& a : g1) {
                if (a.o != (int)o) continue;
                if (j.nin == MAXI) {
                    fail(LDDMM_ERR_DEVICE_CHECK);
                    break;
                }
                j.in[j.nin] = a.buf;
                j.isym[j.nin] = sym(a.scale, a.lpow, a.cls == 0 ? 0 : -1, a.mask);
                j.nin++;
            }
            for (auto& b : outs[o].bases) {
                if (j.nb == MAXB) {
                    fail(LDDMM_ERR_DEVICE_CHECK);
                    break;
                }
                j.base[j.nb] = b.first;
                j.bcoef[j.nb] = b.second;
                j.nb++;
            }
            j0.push_back(j);
        }
        launch(0, -1, j0, bd);
    }

    // comp c of a vector spectral lincomb
    SpecLin lin(std::initializer_list<std::pair<const C*, double>> terms, int c) const {
        SpecLin s;
        s.n = 0;
        for (auto& t : terms) {
            s.p[s.n] = t.first + (size_t)c * d.NS;
            s.c[s.n] = t.second;
            s.n++;
        }
        return s;
    }

    // real vector field (3 comps) -> spectral
    void fwd_vec(const T* in, C* out, double scale = 1.0, int lpow = 0, bool band = false) {
        std::vector<FwdOut> outs(3);
        for (int c = 0; c < 3; ++c) {
            outs[c].out = out + c * d.NS;
            outs[c].terms.push_back({in + c * d.N, sym(scale, lpow, -1)});
        }
        forward(outs, band);
    }
    void inv_vec(const C* in, T* out, int ncomp = 3, bool band = false) {
        std::vector<SpecLin> srcs;
        std::vector<InvReq> reqs;
        for (int c = 0; c < ncomp; ++c) {
            SpecLin s;
            s.n = 1;
            s.p[0] = in + c * d.NS;
            s.c[0] = 1.0;
            srcs.push_back(s);
            reqs.push_back({c, sym(1.0, 0, -1), out + c * d.N});
        }
        inverse(srcs, reqs, band);
    }

    // v, Dv, m = Lv, Dm of a band-limited spectral vector lincomb, into the
    // 24-field layout
    void eval_fields(std::initializer_list<std::pair<const C*, double>> terms, T* S, bool with_m = true) {
        std::vector<SpecLin> srcs;
        std::vector<InvReq> reqs;
        for (int c = 0; c < 3; ++c) srcs.push_back(lin(terms, c));
        for (int c = 0; c < 3; ++c) {
            reqs.push_back({c, sym(1.0, 0, -1), S + c * d.N});
            for (int j = 0; j < 3; ++j) reqs.push_back({c, sym(1.0, 0, j), S + (3 + 3 * c + j) * d.N});
            if (with_m) {
                reqs.push_back({c, sym(1.0, 1, -1), S + (12 + c) * d.N});
                for (int j = 0; j < 3; ++j) reqs.push_back({c, sym(1.0, 1, j), S + (15 + 3 * c + j) * d.N});
            }
        }
        inverse(srcs, reqs, true);
    }

    // ------------------------------------------------------------ reductions
    void dot_async(const T* a, const T* b, size_t n, int slot, double scale) {
        {
            PScope ps_(this, KC_RED, (double)(b ? 2 : 1) * n * sizeof(T));
            k_dot_partial<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, n, partial);
        }
        {
            PScope ps_(this, KC_RED, 0.0);
            k_finish<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 1, 0, 0, scale, dres + slot);
        }
    }
    void minmax_async(const T* a, size_t n, int slot) {  // slots: max|a|, max a, min a
        {
            PScope ps_(this, KC_RED, (double)n * sizeof(T));
            k_absmax_partial<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, n, partial);
        }
        for (int q = 0; q < 3; ++q)
            {
                PScope ps_(this, KC_RED, 0.0);
                k_finish<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 3, q, q == 2 ? 2 : 1, 1.0, dres + slot + q);
            }
    }
    lddmm_status fetch(int first, int count) {
        LD_CK(cudaMemcpyAsync(hres + first, dres + first, count * sizeof(double), cudaMemcpyDeviceToHost, st));
        LD_CK(cudaStreamSynchronize(st));
        return LDDMM_OK;
    }
    double dot_now(const T* a, const T* b, size_t n) {
        dot_async(a, b, n, 63, d.cell);
        if (fetch(63, 1) != LDDMM_OK) return NAN;
        return hres[63];
    }
    lddmm_status check_launch() {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(LDDMM_ERR_CUDA);
        return status;
    }

    // Non-finite input scan (the error convention of the boundary): one
    // launch over the array inputs of a call, whose verdict is copied to
    // pinned host memory at once; scan_verdict() waits for that copy only
    // (not for the call's other work, queued behind it) and makes
    // LDDMM_ERR_NONFINITE sticky.
    void scan_inputs(std::initializer_list<std::pair<const void*, size_t>> arrays) {
        ScanArgs<T> a;
        a.cnt = 0;
        double bytes = 0.0;
        for (const auto& x : arrays) {
            if (!x.first || a.cnt == SCAN_MAX) continue;
            a.p[a.cnt] = (const T*)x.first;
            a.n[a.cnt] = x.second;
            bytes += (double)x.second * sizeof(T);
            a.cnt++;
        }
        if (!a.cnt) return;
        {
            PScope ps_(this, KC_SCAN, bytes);
            k_nonfinite_scan<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, dres + SCAN_SLOT);
        }
        cudaMemcpyAsync(hres + SCAN_SLOT, dres + SCAN_SLOT, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaEventRecord(scan_ev, st);
        scan_pending = true;
    }
    lddmm_status scan_verdict() {
        if (!scan_pending) return status;
        scan_pending = false;
        if (cudaEventSynchronize(scan_ev) != cudaSuccess) return fail(LDDMM_ERR_CUDA);
        if (hres[SCAN_SLOT] != 0.0) return fail(LDDMM_ERR_NONFINITE);
        return status;
    }
    // end of an asynchronous call: launch errors, then the scan's verdict
    lddmm_status finish() {
        if (check_launch() != LDDMM_OK) return status;
        return scan_verdict();
    }

    // One semi-Lagrangian map step u0 -> u1 (velocities v0 at t_k, v1 at
    // t_{k+1}): the shared-memory staged kernel in FP32, the plain gather
    // kernel in FP64 (or if the staged kernel's shared memory was refused).
    void sl_step(const GridI& gi, const T* v0, const T* v1, const T* u0, T* u1, T dt_, T ih0, T ih1, T ih2,
                 int cubic) {
        if constexpr (sizeof(T) == 4) {
            if (sl_staged) {
                const dim3 grid((d.n2 + SLT2 - 1) / SLT2, (d.n1 + SLT1 - 1) / SLT1, (d.n0 + SLT0 - 1) / SLT0);
                if (cubic)
                    k_sl_step_staged<true><<<grid, SLT1 * SLT2, SLBox<true>::SMEM, st>>>(gi, v0, v1, u0, u1, dt_, ih0,
                                                                                          ih1, ih2, d.N);
                else
                    k_sl_step_staged<false><<<grid, SLT1 * SLT2, SLBox<false>::SMEM, st>>>(gi, v0, v1, u0, u1, dt_,
                                                                                            ih0, ih1, ih2, d.N);
                return;
            }
        }
        k_sl_step<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, v0, v1, u0, u1, dt_, ih0, ih1, ih2, cubic, d.N);
    }

    // ------------------------------------------------------------ shooting
    // One Heun step of the EPDiff shooting from `cur` into `nxt`, storing the
    // fields of both stages.  With `transport` the semi-Lagrangian map step
    // k-1 -> k runs too (its velocities are the FP32 copies in vss).
    void shoot_step(int k, const C* cur, C* nxt, bool transport, bool kinetic) {
        const double dt_ = dt();
        const GridI gi{d.n0, d.n1, d.n2};
        const T ih0 = (T)(1.0 / d.h[0]), ih1 = (T)(1.0 / d.h[1]), ih2 = (T)(1.0 / d.h[2]);
        const int cubic = prm.interp == LDDMM_INTERP_CUBIC;
        // Stage fields are evaluated in the compute type: straight into the
        // state store, or into scratch when the store keeps bfloat16 (then
        // k_adstar writes the rounded copy).
        T* a = bf16 ? rs + 24 * d.N : rs;
        const double adb = 27.0 * d.N * sizeof(T) + (bf16 ? 48.0 * d.N : 0.0);
        // stage 1 at v_k
        T* S1 = bf16 ? rs : state(2 * k);
        eval_fields({{cur, 1.0}}, S1);
        if (kinetic) dot_async(S1 + 12 * d.N, S1, 3 * d.N, k, d.cell);
        if (transport && k >= 1) {
            PScope ps_(this, KC_SL, 12.0 * d.N * sizeof(T));
            sl_step(gi, vss[(k - 1) % 2], S1, ubuf_at(k - 1), ubuf_at(k), (T)dt_, ih0, ih1, ih2, cubic);
        }
        {
            PScope ps_(this, KC_ADSTAR, adb);
            k_adstar<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(StatePtr<T>{S1, d.N}, a, d.N,
                                                            bf16 ? state_bf(2 * k) : nullptr);
        }
        if (transport) cudaMemcpyAsync(vss[k % 2], S1, 3 * d.N * sizeof(T), cudaMemcpyDeviceToDevice, st);
        {
            std::vector<FwdOut> outs(3);
            for (int c = 0; c < 3; ++c) {
                outs[c].out = R1 + c * d.NS;
                outs[c].terms.push_back({a + c * d.N, sym(-1.0, -1, -1, 1)});
            }
            forward(outs, true);
        }
        // stage 2 at v*_k = v_k + dt R1
        T* S2 = bf16 ? rs : state(2 * k + 1);
        eval_fields({{cur, 1.0}, {R1, dt_}}, S2);
        {
            PScope ps_(this, KC_ADSTAR, adb);
            k_adstar<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(StatePtr<T>{S2, d.N}, a, d.N,
                                                            bf16 ? state_bf(2 * k + 1) : nullptr);
        }
        {
            std::vector<FwdOut> outs(3);
            for (int c = 0; c < 3; ++c) {
                outs[c].out = nxt + c * d.NS;
                outs[c].terms.push_back({a + c * d.N, sym(-0.5 * dt_, -1, -1, 1)});
                outs[c].bases.push_back({cur + c * d.NS, 1.0});
                outs[c].bases.push_back({R1 + c * d.NS, 0.5 * dt_});
            }
            forward(outs, true);
        }
    }

    // Make the states of segment j resident (checkpointing): re-shoot its
    // steps from the stored spectral velocity of its first step.
    void ensure_segment(int j) {
        if (!ckpt || seg_res == j) return;
        seg_res = j;
        const int k0 = j * cpe, k1 = std::min(prm.nt, k0 + cpe);
        for (int k = k0; k < k1; ++k) {
            const C* cur = k == k0 ? cps + (size_t)j * 3 * d.NS : vhat[k % 2];
            shoot_step(k, cur, vhat[(k + 1) % 2], false, false);
        }
    }

    // v0 real -> stores the stage fields, u1 in ubuf[nt%2], kinetic in dres[0..nt]
    void shoot_core(const T* v0, bool kinetic) {
        NvtxRange nr_("lddmm shoot");
        const double dt_ = dt();
        const int nt = prm.nt;
        const GridI gi{d.n0, d.n1, d.n2};
        const T ih0 = (T)(1.0 / d.h[0]), ih1 = (T)(1.0 / d.h[1]), ih2 = (T)(1.0 / d.h[2]);
        const int cubic = prm.interp == LDDMM_INTERP_CUBIC;
        fwd_vec(v0, v0full);
        mask_copy(v0full, v0hat);
        cudaMemsetAsync(ubuf_at(0), 0, 3 * d.N * sizeof(T), st);
        for (int k = 0; k < nt; ++k) {
            C* cur = k == 0 ? v0hat : vhat[k % 2];
            C* nxt = vhat[(k + 1) % 2];
            if (ckpt && k % cpe == 0) {
                cudaMemcpyAsync(cps + (size_t)(k / cpe) * 3 * d.NS, cur, 3 * d.NS * sizeof(C),
                                cudaMemcpyDeviceToDevice, st);
                seg_res = k / cpe;
            }
            shoot_step(k, cur, nxt, true, kinetic);
        }
        // v_nt, m_nt in real space, last map step
        {
            std::vector<SpecLin> srcs;
            std::vector<InvReq> reqs;
            for (int c = 0; c < 3; ++c) {
                SpecLin s;
                s.n = 1;
                s.p[0] = vhat[nt % 2] + c * d.NS;
                s.c[0] = 1.0;
                srcs.push_back(s);
                reqs.push_back({c, sym(1.0, 0, -1), vfin + c * d.N});
                reqs.push_back({c, sym(1.0, 1, -1), vfin + (3 + c) * d.N});
            }
            inverse(srcs, reqs, true);
        }
        if (kinetic) dot_async(vfin + 3 * d.N, vfin, 3 * d.N, nt, d.cell);
        {
            PScope ps_(this, KC_SL, 12.0 * d.N * sizeof(T));
            sl_step(gi, vss[(nt - 1) % 2], vfin, ubuf_at(nt - 1), ubuf_at(nt), (T)dt_, ih0, ih1, ih2, cubic);
        }
    }
    T* u1() const { return ubuf_at(prm.nt); }

    void warp_and_grad(const T* I0) {
        const GridI gi{d.n0, d.n1, d.n2};
        {
            PScope ps_(this, KC_WARP, 5.0 * d.N * sizeof(T));
            k_warp<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, I0, u1(), m1, (T)(1.0 / d.h[0]), (T)(1.0 / d.h[1]),
                                                          (T)(1.0 / d.h[2]), prm.interp == LDDMM_INTERP_CUBIC, d.N);
        }
        std::vector<FwdOut> outs(1);
        outs[0].out = tmp;
        outs[0].terms.push_back({m1, sym(1.0, 0, -1)});
        forward(outs);
        std::vector<SpecLin> srcs(1);
        srcs[0].n = 1;
        srcs[0].p[0] = tmp;
        srcs[0].c[0] = 1.0;
        std::vector<InvReq> reqs;
        for (int j = 0; j < 3; ++j) reqs.push_back({0, sym(1.0, 0, j), gm1 + j * d.N});
        inverse(srcs, reqs);
    }

    // ------------------------------------------------------------ Jacobi sweeps
    // tangent: from tan_[0] = (eta0, xi0); result in tan_[nt % 2]
    void tangent_sweep() {
        NvtxRange nr_("lddmm tangent sweep");
        const double dt_ = dt();
        T* E = rs;                  // 24 fields
        T* X = rs + 24 * d.N;       // 12 fields
        T* pq_ = rs + 36 * d.N;     // 6 fields
        for (int k = 0; k < prm.nt; ++k) {
            ensure_segment(k / cpe);
            C* cur = tan_[k % 2];
            C* nxt = tan_[(k + 1) % 2];
            C* ce = cur;
            C* cx = cur + 3 * d.NS;
            C* be = tb;
            C* bx = tb + 3 * d.NS;
            for (int stg = 0; stg < 2; ++stg) {
                const int sidx = 2 * k + stg;
                std::vector<SpecLin> srcs;
                std::vector<InvReq> reqs;
                for (int c = 0; c < 3; ++c) {
                    if (stg == 0) srcs.push_back(lin({{ce, 1.0}}, c));
                    else srcs.push_back(lin({{ce, 1.0}, {be, dt_}}, c));
                }
                for (int c = 0; c < 3; ++c) {
                    if (stg == 0) srcs.push_back(lin({{cx, 1.0}}, c));
                    else srcs.push_back(lin({{cx, 1.0}, {bx, dt_}}, c));
                }
                for (int c = 0; c < 3; ++c) {
                    reqs.push_back({c, sym(1.0, 0, -1), E + c * d.N});
                    for (int j = 0; j < 3; ++j) reqs.push_back({c, sym(1.0, 0, j), E + (3 + 3 * c + j) * d.N});
                    reqs.push_back({c, sym(1.0, 1, -1), E + (12 + c) * d.N});
                    for (int j = 0; j < 3; ++j) reqs.push_back({c, sym(1.0, 1, j), E + (15 + 3 * c + j) * d.N});
                    reqs.push_back({3 + c, sym(1.0, 0, -1), X + c * d.N});
                    for (int j = 0; j < 3; ++j) reqs.push_back({3 + c, sym(1.0, 0, j), X + (3 + 3 * c + j) * d.N});
                }
                std::vector<FwdOut> outs(6);
                for (int c = 0; c < 3; ++c) {
                    FwdOut& oe = outs[c];
                    FwdOut& ox = outs[3 + c];
                    if (stg == 0) {
                        oe.out = be + c * d.NS;
                        oe.terms.push_back({pq_ + c * d.N, sym(-1.0, -1, -1, 1)});
                        ox.out = bx + c * d.NS;
                        ox.terms.push_back({pq_ + (3 + c) * d.N, sym(1.0, 0, -1, 1)});
                        ox.bases.push_back({ce + c * d.NS, 1.0});
                    } else {
                        oe.out = nxt + c * d.NS;
                        oe.terms.push_back({pq_ + c * d.N, sym(-0.5 * dt_, -1, -1, 1)});
                        oe.bases.push_back({ce + c * d.NS, 1.0});
                        oe.bases.push_back({be + c * d.NS, 0.5 * dt_});
                        ox.out = nxt + (3 + c) * d.NS;
                        ox.terms.push_back({pq_ + (3 + c) * d.N, sym(0.5 * dt_, 0, -1, 1)});
                        ox.bases.push_back({cx + c * d.NS, 1.0});
                        ox.bases.push_back({bx + c * d.NS, 0.5 * dt_});
                        ox.bases.push_back({ce + c * d.NS, 0.5 * dt_});
                        ox.bases.push_back({be + c * d.NS, 0.5 * dt_ * dt_});
                    }
                }
                if (fused) {
                    tangent_stage_fused(srcs, reqs, outs, sidx);
                    continue;
                }
                inverse(srcs, reqs, true);
                {
                    PScope ps_(this, KC_TANPW, 24.0 * d.N * state_elem() + 42.0 * d.N * sizeof(T));
                    if (bf16)
                        k_tangent_pw<T, __nv_bfloat16><<<pw_grid(d.N), PW_THREADS, 0, st>>>(
                            StatePtr<__nv_bfloat16>{state_bf(sidx), d.N}, StatePtr<T>{E, d.N}, X, pq_, d.N);
                    else
                        k_tangent_pw<T, T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(StatePtr<T>{state(sidx), d.N},
                                                                               StatePtr<T>{E, d.N}, X, pq_, d.N);
                }
                forward(outs, true);
            }
        }
    }

    // ---- fused Jacobi stages (FP32): axis-0/1 passes of the inverse transform,
    // one fused kernel (axis-2 inverse, pointwise products, axis-2 forward),
    // axis-1/0 passes of the forward transform
    void fused_launch(FusedArgs& a, int sidx, int kind) {
        if constexpr (sizeof(T) == 4) {
            a.states = bf16 ? (const void*)state_bf(sidx) : (const void*)state(sidx);
            a.dk2 = (const float*)tabs.dk[2];
            a.tw = (const cpx<float>*)ax[2].tw;
            a.rows = (int)d.rows;
            a.nb2 = bnb2;
            a.ntiles = (int)(d.rows / (size_t)FusedPass::tile_rows(d.n2));
            a.npts = (unsigned)d.N;
            const double band = (double)bnb2 * d.rows * sizeof(C);
            const double bytes = 33.0 * band + 24.0 * d.N * state_elem() + (a.eta_src ? 3.0 * d.N * sizeof(T) : 0.0);
            PScope ps_(this, kind == 0 ? KC_TANF : KC_ADJF, bytes);
            bool ok;
            if (bf16) {
                if (kind == 0) ok = FusedPass::launch<__nv_bfloat16, 0>(d.n2, a, st);
                else ok = FusedPass::launch<__nv_bfloat16, 1>(d.n2, a, st);
            } else {
                if (kind == 0) ok = FusedPass::launch<float, 0>(d.n2, a, st);
                else ok = FusedPass::launch<float, 1>(d.n2, a, st);
            }
            if (!ok) fail(LDDMM_ERR_DEVICE_CHECK);
        }
    }
    // tangent stage: requests per component c (12 c + ...): eta, D_j eta (3),
    // mu, D_j mu (3), xi, D_j xi (3); outputs p_0..2, q_0..2
    void tangent_stage_fused(const std::vector<SpecLin>& srcs, const std::vector<InvReq>& reqs,
                             const std::vector<FwdOut>& outs, int sidx) {
        const InvHead ih = inverse_head(srcs, reqs, true);
        FusedArgs a;
        memset(&a, 0, sizeof(a));
        auto k1 = [&](int r) { return (const cpx<float>*)ih.k1[ih.r1[r]]; };
        for (int c = 0; c < 3; ++c) {
            const int r = 12 * c;
            // each D2 field reads the spectrum of its plain field
            for (int q : {0, 4, 8})
                if (ih.r1[r + q + 3] != ih.r1[r + q] || !ih.d2[r + q + 3] || ih.d2[r + q]) {
                    fail(LDDMM_ERR_DEVICE_CHECK);
                    return;
                }
            a.in[6 * c + 0] = k1(r);
            a.in[6 * c + 1] = k1(r + 1);
            a.in[6 * c + 2] = k1(r + 2);
            a.in[6 * c + 3] = k1(r + 4);
            a.in[6 * c + 4] = k1(r + 5);
            a.in[6 * c + 5] = k1(r + 6);
            a.in[18 + 3 * c] = k1(r + 8);
            a.in[19 + 3 * c] = k1(r + 9);
            a.in[20 + 3 * c] = k1(r + 10);
        }
        std::vector<G> g2;
        for (int o = 0; o < 6; ++o) {
            const SymD& sy = outs[o].terms[0].sym;
            g2.push_back({o, sy.lpow, sy.scale, 2, 1, palloc(), 1});
            a.out[o] = (cpx<float>*)g2.back().buf;
        }
        fused_launch(a, sidx, 0);
        forward_tail(outs, g2, true);
    }
    // adjoint stage: requests (K ybar_eta_c, P ybar_xi_c) for c = 0..2;
    // outputs per c: groups (s, f) of R'^T without L and under -L into eta_c,
    // of ad_v^T into xi_c, each as (cls 2, cls 0, cls 1) partial spectra
    void adjoint_stage_fused(const std::vector<SpecLin>& srcs, const std::vector<InvReq>& reqs,
                             const std::vector<FwdOut>& outs, int sidx, const T* eta) {
        const InvHead ih = inverse_head(srcs, reqs, true);
        FusedArgs a;
        memset(&a, 0, sizeof(a));
        for (int c = 0; c < 3; ++c) {
            if (ih.d2[2 * c] || ih.d2[2 * c + 1]) {
                fail(LDDMM_ERR_DEVICE_CHECK);
                return;
            }
            a.in[c] = (const cpx<float>*)ih.k1[ih.r1[2 * c]];
            a.in[3 + c] = (const cpx<float>*)ih.k1[ih.r1[2 * c + 1]];
        }
        std::vector<G> g2;
        for (int c = 0; c < 3; ++c)
            for (int g = 0; g < 3; ++g)
                for (int cls : {2, 0, 1}) {
                    g2.push_back({g < 2 ? c : 3 + c, g == 1 ? 1 : 0, g == 1 ? -1.0 : 1.0, cls, 1, palloc(), 1});
                    a.out[g2.size() - 1] = (cpx<float>*)g2.back().buf;
                }
        a.eta_src = (const float*)eta;
        fused_launch(a, sidx, 1);
        forward_tail(outs, g2, true);
    }

    // adjoint: from adj[0] = (ybar_eta, ybar_xi) at t = 1; result in adj[nt % 2].
    // eta_src (nullable): real cotangents on eta_k, k = 0..nt (3 fields each),
    // added to ybar_eta after the transposed step k (exact discrete gradient)
    void adjoint_sweep(const T* eta_src = nullptr) {
        NvtxRange nr_("lddmm adjoint sweep");
        const double dt_ = dt();
        T* Y = rs;              // 6 fields
        T* G = rs + 6 * d.N;    // 36 fields
        int cur_i = 0;
        for (int k = prm.nt - 1; k >= 0; --k) {
            ensure_segment(k / cpe);
            C* cur = adj[cur_i];
            C* nxt = adj[1 - cur_i];
            C* ce = cur;
            C* cx = cur + 3 * d.NS;
            C* ae = adja;
            C* axp = adja + 3 * d.NS;
            for (int stg = 0; stg < 2; ++stg) {
                const int sidx = stg == 0 ? 2 * k + 1 : 2 * k;
                std::vector<SpecLin> srcs;
                std::vector<InvReq> reqs;
                for (int c = 0; c < 3; ++c) {
                    if (stg == 0) srcs.push_back(lin({{ce, 1.0}}, c));
                    else srcs.push_back(lin({{ce, 0.5 * dt_}, {ae, 0.5 * dt_ * dt_}}, c));
                }
                for (int c = 0; c < 3; ++c) {
                    if (stg == 0) srcs.push_back(lin({{cx, 1.0}}, c));
                    else srcs.push_back(lin({{cx, 0.5 * dt_}, {axp, 0.5 * dt_ * dt_}}, c));
                }
                for (int c = 0; c < 3; ++c) {
                    reqs.push_back({c, sym(1.0, -1, -1, 1), Y + c * d.N});
                    reqs.push_back({3 + c, sym(1.0, 0, -1, 1), Y + (3 + c) * d.N});
                }
                std::vector<FwdOut> outs(6);
                for (int c = 0; c < 3; ++c) {
                    FwdOut& oe = outs[c];
                    FwdOut& ox = outs[3 + c];
                    const T* g1 = G + (size_t)(4 * c) * d.N;
                    const T* g2 = G + (size_t)(4 * (3 + c)) * d.N;
                    const T* g3 = G + (size_t)(4 * (6 + c)) * d.N;
                    oe.terms.push_back({g1, sym(1.0, 0, -1)});
                    oe.terms.push_back({g2, sym(-1.0, 1, -1)});
                    ox.terms.push_back({g3, sym(1.0, 0, -1)});
                    for (int j = 0; j < 3; ++j) {
                        oe.terms.push_back({g1 + (1 + j) * d.N, sym(1.0, 0, j)});
                        oe.terms.push_back({g2 + (1 + j) * d.N, sym(-1.0, 1, j)});
                        ox.terms.push_back({g3 + (1 + j) * d.N, sym(1.0, 0, j)});
                    }
                    if (stg == 0) {
                        oe.out = ae + c * d.NS;
                        oe.bases.push_back({cx + c * d.NS, 1.0});
                        ox.out = axp + c * d.NS;
                    } else {
                        oe.out = nxt + c * d.NS;
                        oe.bases.push_back({ce + c * d.NS, 1.0});
                        oe.bases.push_back({ae + c * d.NS, 0.5 * dt_});
                        oe.bases.push_back({cx + c * d.NS, 0.5 * dt_});
                        oe.bases.push_back({axp + c * d.NS, 0.5 * dt_ * dt_});
                        if (eta_src) oe.terms.push_back({eta_src + ((size_t)3 * k + c) * d.N, sym(1.0, 0, -1)});
                        ox.out = nxt + (3 + c) * d.NS;
                        ox.bases.push_back({cx + c * d.NS, 1.0});
                        ox.bases.push_back({axp + c * d.NS, 0.5 * dt_});
                    }
                }
                if (fused) {
                    adjoint_stage_fused(srcs, reqs, outs, sidx,
                                        stg == 1 && eta_src ? eta_src + (size_t)3 * k * d.N : nullptr);
                    continue;
                }
                inverse(srcs, reqs, true);
                {
                    PScope ps_(this, KC_ADJPW, 24.0 * d.N * state_elem() + 42.0 * d.N * sizeof(T));
                    if (bf16)
                        k_adjoint_pw<T, __nv_bfloat16><<<pw_grid(d.N), PW_THREADS, 0, st>>>(
                            StatePtr<__nv_bfloat16>{state_bf(sidx), d.N}, Y, G, d.N);
                    else
                        k_adjoint_pw<T, T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(StatePtr<T>{state(sidx), d.N}, Y, G, d.N);
                }
                forward(outs, true);
            }
            cur_i = 1 - cur_i;
        }
    }
    C* adj_result() const { return adj[prm.nt % 2]; }

    // spectral out (3) = a_sym . A + b_sym . B  -> real
    void spec_to_real2(const C* A, SymD sa, const C* B, SymD sb, T* out) {
        for (int c = 0; c < 3; ++c) {
            SpecComb<T> sc;
            sc.nin = 0;
            if (A) {
                sc.in[sc.nin] = A + c * d.NS;
                sc.sym[sc.nin++] = to_symt<T>(sa);
            }
            if (B) {
                sc.in[sc.nin] = B + c * d.NS;
                sc.sym[sc.nin++] = to_symt<T>(sb);
            }
            {
                PScope ps_(this, KC_SPEC, (double)(sc.nin + 1) * d.NS * sizeof(C));
                k_spec_comb<T><<<spec_comb_blocks(d.n0, d.n2h), spec_comb_threads(d.n1), 0, st>>>(sc, tabs, d.n0, d.n1,
                                                                                               d.n2h, tmp + c * d.NS);
            }
        }
        inv_vec(tmp, out);
    }

    // Exact discrete gradient, transport part: dE_data/dv_k (k = 0..nt) into
    // vbar through the transposes of the warp and of the map steps, backwards
    // from t = 1 (needs the maps u_k of the last shoot and m1).
    void exact_data_cotangents(const T* I0, const T* I1) {
        const GridI gi{d.n0, d.n1, d.n2};
        const T ih0 = (T)(1.0 / d.h[0]), ih1 = (T)(1.0 / d.h[1]), ih2 = (T)(1.0 / d.h[2]);
        const int cubic = prm.interp == LDDMM_INTERP_CUBIC;
        const int nt = prm.nt;
        cudaMemsetAsync(vbar, 0, (size_t)3 * (nt + 1) * d.N * sizeof(T), st);
        {
            PScope ps_(this, KC_WARP, 8.0 * d.N * sizeof(T));
            if (cubic)
                k_warp_adj<T, true><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, I0, u1(), m1, I1, ubar[0], ih0, ih1, ih2,
                                                                        d.N);
            else
                k_warp_adj<T, false><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, I0, u1(), m1, I1, ubar[0], ih0, ih1,
                                                                         ih2, d.N);
        }
        int cu = 0;
        for (int k = nt - 1; k >= 0; --k) {
            cudaMemsetAsync(ubar[1 - cu], 0, 3 * d.N * sizeof(T), st);
            const T* vk = state(2 * k);                            // stage-1 velocity v_k
            const T* vk1 = k + 1 == nt ? vfin : state(2 * (k + 1));  // v_{k+1}
            {
                PScope ps_(this, KC_SL, 24.0 * d.N * sizeof(T));
                T* vb0 = vbar + (size_t)3 * k * d.N;
                T* vb1 = vbar + (size_t)3 * (k + 1) * d.N;
                if (cubic)
                    k_sl_adj<T, true><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, vk, vk1, ubuf_at(k), ubar[cu],
                                                                          ubar[1 - cu], vb0, vb1, (T)dt(), ih0, ih1,
                                                                          ih2, d.N);
                else
                    k_sl_adj<T, false><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, vk, vk1, ubuf_at(k), ubar[cu],
                                                                           ubar[1 - cu], vb0, vb1, (T)dt(), ih0, ih1,
                                                                           ih2, d.N);
            }
            cu = 1 - cu;
        }
    }

    // gradient internals: E into dres[nt+1..nt+3]; gradient real in metric `space`
    void gradient_core(const T* v0, const T* I0, const T* I1, T* grad, int space) {
        NvtxRange nr_("lddmm gradient");
        shoot_core(v0, true);
        warp_and_grad(I0);
        {
            PScope ps_(this, KC_MISC, 3.0 * d.N * sizeof(T));
            k_sub<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(m1, I1, rbuf, d.N);
        }
        dot_async(rbuf, nullptr, d.N, prm.nt + 2, d.cell);
        reg_async(v0, prm.nt + 1);
        if (exact_grad) {
            exact_data_cotangents(I0, I1);
            // eta block from dE/dv_nt, xi block zero; dE/dv_k enter along the way
            fwd_vec(vbar + (size_t)3 * prm.nt * d.N, adj[0], 1.0, 0, true);
            cudaMemsetAsync(adj[0] + 3 * d.NS, 0, 3 * d.NS * sizeof(C), st);
            adjoint_sweep(vbar);
        } else {
            {
                PScope ps_(this, KC_MISC, 8.0 * d.N * sizeof(T));
                k_final_source<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(m1, I1, gm1, nullptr, rs, 0, d.N);
            }
            fwd_vec(rs, adj[0] + 3 * d.NS, 1.0, 0, true);
            cudaMemsetAsync(adj[0], 0, 3 * d.NS * sizeof(C), st);
            adjoint_sweep();
        }
        // g_L2 = 2 w L v0 + T^T b ;  V: K g_L2 = 2 w v0 + K T^T b
        const double w2 = 2.0 * prm.weight;
        if (space == LDDMM_SPACE_V)
            spec_to_real2(v0full, sym(w2, 0, -1), adj_result(), sym(1.0, -1, -1, 1), grad);
        else
            spec_to_real2(v0full, sym(w2, 1, -1), adj_result(), sym(1.0, 0, -1, 1), grad);
        lin_valid = true;
    }
    // ---- the Hessian-vector product as a CUDA graph.  Its ~220 launches
    // depend only on the handle and on (dv0, out, space): they are recorded
    // once (stream capture) and replayed, which removes the gaps between
    // back-to-back launches.  Not with the profiler on (it times each
    // launch), with checkpointed states (the re-shooting depends on which
    // segment is resident), or when the stream cannot be captured (the
    // legacy default stream): then the kernels are launched one by one.
    struct HvGraph {
        const void* in = nullptr;
        void* out = nullptr;
        int space = -1;
        cudaGraphExec_t exec = nullptr;
    };
    HvGraph hvg;
    void hessvec_run(const T* dv0, T* out, int space) {
        if (prof_on || ckpt || force_no_graph()) {
            hessvec_core(dv0, out, space);
            return;
        }
        if (!(hvg.exec && hvg.in == dv0 && hvg.out == out && hvg.space == space)) {
            if (hvg.exec) {
                cudaGraphExecDestroy(hvg.exec);
                hvg.exec = nullptr;
            }
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                hessvec_core(dv0, out, space);
                return;
            }
            hessvec_core(dv0, out, space);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess || !g || cudaGraphInstantiate(&hvg.exec, g, 0) != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                hvg.exec = nullptr;
                cudaGetLastError();
                hessvec_core(dv0, out, space);  // the captured launches did not run
                return;
            }
            cudaGraphDestroy(g);
            hvg.in = dv0;
            hvg.out = out;
            hvg.space = space;
        }
        if (cudaGraphLaunch(hvg.exec, st) != cudaSuccess) fail(LDDMM_ERR_CUDA);
    }

    void hessvec_core(const T* dv0, T* out, int space) {
        NvtxRange nr_("lddmm hessvec");
        fwd_vec(dv0, dhat);
        mask_copy(dhat, tan_[0]);
        cudaMemsetAsync(tan_[0] + 3 * d.NS, 0, 3 * d.NS * sizeof(C), st);
        tangent_sweep();
        T* xi = rs;
        inv_vec(tan_[prm.nt % 2] + 3 * d.NS, xi, 3, true);
        T* c = rs + 3 * d.N;
        {
            PScope ps_(this, KC_MISC, 8.0 * d.N * sizeof(T));
            k_final_source<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(m1, nullptr, gm1, xi, c, 1, d.N);
        }
        fwd_vec(c, adj[0] + 3 * d.NS, 1.0, 0, true);
        cudaMemsetAsync(adj[0], 0, 3 * d.NS * sizeof(C), st);
        adjoint_sweep();
        const double w2 = 2.0 * prm.weight;
        if (space == LDDMM_SPACE_V)
            spec_to_real2(dhat, sym(w2, 0, -1), adj_result(), sym(1.0, -1, -1, 1), out);
        else
            spec_to_real2(dhat, sym(w2, 1, -1), adj_result(), sym(1.0, 0, -1, 1), out);
    }

    // ------------------------------------------------------------ ABI operations
    lddmm_status shoot(const void* v0, const void* I0, void* m1o, void* u1o, double* kinetic) override {
        if (status != LDDMM_OK) return status;
        if (!v0 || (m1o && !I0)) return fail(LDDMM_ERR_ARG);
        scan_inputs({{v0, 3 * d.N}, {I0, d.N}});
        shoot_core((const T*)v0, kinetic != nullptr);
        lin_valid = false;
        if (I0) {
            // m1 and grad m1 make this shoot a linearisation point (lddmm_shoot_vjp, hessvec)
            warp_and_grad((const T*)I0);
            if (m1o) cudaMemcpyAsync(m1o, m1, d.N * sizeof(T), cudaMemcpyDeviceToDevice, st);
            lin_valid = true;
        }
        if (u1o) cudaMemcpyAsync(u1o, u1(), 3 * d.N * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (finish() != LDDMM_OK) return status;
        if (kinetic) {
            if (fetch(0, prm.nt + 1) != LDDMM_OK) return status;
            for (int k = 0; k <= prm.nt; ++k) kinetic[k] = hres[k];
        }
        return status;
    }

    lddmm_status gradient(const void* v0, const void* I0, const void* I1, void* grad, double* energy) override {
        if (status != LDDMM_OK) return status;
        if (!v0 || !I0 || !I1 || !grad) return fail(LDDMM_ERR_ARG);
        scan_inputs({{v0, 3 * d.N}, {I0, d.N}, {I1, d.N}});
        gradient_core((const T*)v0, (const T*)I0, (const T*)I1, (T*)grad, prm.space);
        if (finish() != LDDMM_OK) return status;
        if (energy) {
            if (fetch(0, prm.nt + 3) != LDDMM_OK) return status;
            const double data = hres[prm.nt + 2], reg = prm.weight * hres[prm.nt + 1];
            energy[0] = data + reg;
            energy[1] = data;
            energy[2] = reg;
            if (!std::isfinite(energy[0])) return fail(LDDMM_ERR_NONFINITE);
        }
        return status;
    }

    lddmm_status hessvec(const void* dv0, void* Hdv) override {
        if (status != LDDMM_OK) return status;
        if (!dv0 || !Hdv) return fail(LDDMM_ERR_ARG);
        if (!lin_valid) return LDDMM_ERR_NOT_LINEARIZED;
        scan_inputs({{dv0, 3 * d.N}});
        hessvec_run((const T*)dv0, (T*)Hdv, prm.space);
        return finish();
    }

    lddmm_status jacobi_forward(const void* dv0, void* eta1, void* xi1) override {
        if (status != LDDMM_OK) return status;
        if (!dv0) return fail(LDDMM_ERR_ARG);
        if (!lin_valid) return LDDMM_ERR_NOT_LINEARIZED;
        scan_inputs({{dv0, 3 * d.N}});
        fwd_vec((const T*)dv0, dhat);
        mask_copy(dhat, tan_[0]);
        cudaMemsetAsync(tan_[0] + 3 * d.NS, 0, 3 * d.NS * sizeof(C), st);
        tangent_sweep();
        if (eta1) inv_vec(tan_[prm.nt % 2], (T*)eta1, 3, true);
        if (xi1) inv_vec(tan_[prm.nt % 2] + 3 * d.NS, (T*)xi1, 3, true);
        return finish();
    }

    lddmm_status jacobi_adjoint(const void* beta, const void* bxi, void* out) override {
        if (status != LDDMM_OK) return status;
        if (!bxi || !out) return fail(LDDMM_ERR_ARG);
        if (!lin_valid) return LDDMM_ERR_NOT_LINEARIZED;
        scan_inputs({{beta, 3 * d.N}, {bxi, 3 * d.N}});
        fwd_vec((const T*)bxi, adj[0] + 3 * d.NS, 1.0, 0, true);
        if (beta) fwd_vec((const T*)beta, adj[0], 1.0, 0, true);
        else cudaMemsetAsync(adj[0], 0, 3 * d.NS * sizeof(C), st);
        adjoint_sweep();
        spec_to_real2(nullptr, sym(0.0, 0, -1), adj_result(), sym(1.0, 0, -1, 1), (T*)out);
        return finish();
    }

    lddmm_status apply_metric(const void* in, void* out, int ncomp, int power) override {
        if (status != LDDMM_OK) return status;
        if (!in || !out || ncomp < 1 || power < -4 || power > 4) return fail(LDDMM_ERR_ARG);
        scan_inputs({{in, (size_t)ncomp * d.N}});
        for (int c0 = 0; c0 < ncomp; c0 += 3) {
            const int nc = std::min(3, ncomp - c0);
            std::vector<FwdOut> outs(nc);
            for (int c = 0; c < nc; ++c) {
                outs[c].out = tmp + c * d.NS;
                outs[c].terms.push_back({(const T*)in + (size_t)(c0 + c) * d.N, sym(1.0, power, -1)});
            }
            forward(outs);
            inv_vec(tmp, (T*)out + (size_t)c0 * d.N, nc);
        }
        return finish();
    }

    void jacdet_into(const T* u, T* J) {
        fwd_vec(u, tmp);
        std::vector<SpecLin> srcs;
        std::vector<InvReq> reqs;
        for (int c = 0; c < 3; ++c) {
            SpecLin s;
            s.n = 1;
            s.p[0] = tmp + c * d.NS;
            s.c[0] = 1.0;
            srcs.push_back(s);
            for (int j = 0; j < 3; ++j) reqs.push_back({c, sym(1.0, 0, j), rs + (3 * c + j) * d.N});
        }
        inverse(srcs, reqs);
        {
            PScope ps_(this, KC_MISC, 10.0 * d.N * sizeof(T));
            k_jacdet<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(rs, J, d.N);
        }
    }

    lddmm_status jacobian_det(const void* u, void* J, double* minmax) override {
        if (status != LDDMM_OK) return status;
        if (!u) return fail(LDDMM_ERR_ARG);
        scan_inputs({{u, 3 * d.N}});
        T* Jd = J ? (T*)J : rs + 9 * d.N;
        jacdet_into((const T*)u, Jd);
        if (minmax) minmax_async(Jd, d.N, 60);
        if (finish() != LDDMM_OK) return status;
        if (minmax) {
            if (fetch(60, 3) != LDDMM_OK) return status;
            minmax[0] = hres[62];
            minmax[1] = hres[61];
        }
        return status;
    }

    // out = T^T (-G grad m1): the vector-Jacobian product of v0 -> m1 at the
    // last linearisation point (Jacobi-field linearisation delta m1 = -grad m1 . xi1)
    lddmm_status shoot_vjp(const void* G, void* out) override {
        if (status != LDDMM_OK) return status;
        if (!G || !out) return fail(LDDMM_ERR_ARG);
        if (!lin_valid) return LDDMM_ERR_NOT_LINEARIZED;
        scan_inputs({{G, d.N}});
        {
            PScope ps_(this, KC_MISC, 8.0 * d.N * sizeof(T));
            k_vjp_source<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>((const T*)G, gm1, rs, d.N);
        }
        fwd_vec(rs, adj[0] + 3 * d.NS, 1.0, 0, true);
        cudaMemsetAsync(adj[0], 0, 3 * d.NS * sizeof(C), st);
        adjoint_sweep();
        spec_to_real2(nullptr, sym(0.0, 0, -1), adj_result(), sym(1.0, 0, -1, 1), (T*)out);
        return finish();
    }

    lddmm_status synchronize() override {
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(LDDMM_ERR_CUDA);
        return check_launch();
    }

    // ------------------------------------------------------------ GN-Krylov
    double energy_at(const T* v, const T* I0, const T* I1) {
        shoot_core(v, true);
        lin_valid = false;
        const GridI gi{d.n0, d.n1, d.n2};
        {
            PScope ps_(this, KC_WARP, 5.0 * d.N * sizeof(T));
            k_warp<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(gi, I0, u1(), m1, (T)(1.0 / d.h[0]), (T)(1.0 / d.h[1]),
                                                          (T)(1.0 / d.h[2]), prm.interp == LDDMM_INTERP_CUBIC, d.N);
        }
        {
            PScope ps_(this, KC_MISC, 3.0 * d.N * sizeof(T));
            k_sub<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(m1, I1, rbuf, d.N);
        }
        dot_async(rbuf, nullptr, d.N, prm.nt + 2, d.cell);
        reg_async(v, prm.nt + 1);
        if (fetch(0, prm.nt + 3) != LDDMM_OK) return NAN;
        return hres[prm.nt + 2] + prm.weight * hres[prm.nt + 1];
    }

    void kapply(const T* in, T* out) {  // out = K in (3 comps)
        fwd_vec(in, tmp, 1.0, -1);
        inv_vec(tmp, out);
    }

    lddmm_status reg(const void* I0v, const void* I1v, void* v0v, lddmm_report* rep) override {
        if (status != LDDMM_OK) return status;
        if (!I0v || !I1v || !v0v) return fail(LDDMM_ERR_ARG);
        scan_inputs({{I0v, d.N}, {I1v, d.N}, {v0v, 3 * d.N}});
        if (scan_verdict() != LDDMM_OK) return status;
        const T* I0 = (const T*)I0v;
        const T* I1 = (const T*)I1v;
        T* v = (T*)v0v;
        const size_t n3 = 3 * d.N;
        const int g = pw_grid(n3);
        lddmm_report R;
        memset(&R, 0, sizeof(R));
        double g0max = 0.0;
        bool ls_fail = false;
        const int maxit = std::min(prm.gn_maxit, LDDMM_TRACE_MAX);
        int it = 0;
        double eps_prev = 0.0;
        for (; it < maxit && prm.optimizer == LDDMM_OPT_GD; ++it) {
            // gradient descent in V (Sec. 2.2): v0 <- v0 - eps K g_L2
            gradient_core(v, I0, I1, pg, LDDMM_SPACE_L2);
            if (fetch(0, prm.nt + 3) != LDDMM_OK) return status;
            const double E = hres[prm.nt + 2] + prm.weight * hres[prm.nt + 1];
            if (!std::isfinite(E)) return fail(LDDMM_ERR_NONFINITE);
            R.energy[it] = E;
            kapply(pg, pz);
            minmax_async(pz, n3, 60);
            if (fetch(60, 1) != LDDMM_OK) return status;
            const double kgmax = hres[60];  // max |K g_L2|: sets the first trial step
            double gmax = kgmax;            // |g|_inf in the chosen metric
            if (prm.space == LDDMM_SPACE_L2) {
                minmax_async(pg, n3, 60);
                if (fetch(60, 1) != LDDMM_OK) return status;
                gmax = hres[60];
            }
            if (it == 0) g0max = gmax;
            {
                PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                k_lincomb2<T><<<g, PW_THREADS, 0, st>>>((T)-1, pz, (T)0, pz, px, n3);
            }
            const double slope = dot_now(pg, px, n3);
            const double hmin = std::min(d.h[0], std::min(d.h[1], d.h[2]));
            double eps = it == 0 ? (kgmax > 0 ? hmin / kgmax : 1.0) : 2.0 * eps_prev;
            bool ok = false;
            for (int t = 0; t < prm.ls_maxit; ++t) {
                {
                    PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                    k_lincomb2<T><<<g, PW_THREADS, 0, st>>>((T)1, v, (T)eps, px, pvt, n3);
                }
                const double Et = energy_at(pvt, I0, I1);
                if (status != LDDMM_OK) return status;
                if (std::isfinite(Et) && Et <= E + prm.armijo_c1 * eps * slope) {
                    ok = true;
                    break;
                }
                eps *= 0.5;
            }
            R.pcg_iters[it] = 0;
            R.step[it] = ok ? eps : 0.0;
            if (!ok) {
                ls_fail = true;
                ++it;
                break;
            }
            eps_prev = eps;
            cudaMemcpyAsync(v, pvt, n3 * sizeof(T), cudaMemcpyDeviceToDevice, st);
        }
        for (; it < maxit && prm.optimizer == LDDMM_OPT_GN; ++it) {
            gradient_core(v, I0, I1, pg, LDDMM_SPACE_L2);
            if (fetch(0, prm.nt + 3) != LDDMM_OK) return status;
            const double E = hres[prm.nt + 2] + prm.weight * hres[prm.nt + 1];
            if (!std::isfinite(E)) return fail(LDDMM_ERR_NONFINITE);
            R.energy[it] = E;
            // |g|_inf in the chosen metric
            const T* gsp = pg;
            if (prm.space == LDDMM_SPACE_V) {
                kapply(pg, pz);
                gsp = pz;
            }
            minmax_async(gsp, n3, 60);
            if (fetch(60, 1) != LDDMM_OK) return status;
            if (it == 0) g0max = hres[60];
            // PCG on H x = -g, preconditioner K, x0 = 0
            cudaMemsetAsync(px, 0, n3 * sizeof(T), st);
            {
                PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                k_lincomb2<T><<<g, PW_THREADS, 0, st>>>((T)-1, pg, (T)0, pg, pr, n3);
            }
            kapply(pr, pz);
            cudaMemcpyAsync(pp, pz, n3 * sizeof(T), cudaMemcpyDeviceToDevice, st);
            double rz = dot_now(pr, pz, n3);
            const double nrm0 = prm.space == LDDMM_SPACE_V ? std::sqrt(std::max(rz, 0.0)) : std::sqrt(dot_now(pr, pr, n3));
            int pit = 0;
            while (pit < prm.pcg_maxit) {
                hessvec_run(pp, pq, LDDMM_SPACE_L2);
                const double pq_ = dot_now(pp, pq, n3);
                if (!(pq_ > 0.0)) break;
                const double alpha = rz / pq_;
                {
                    PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                    k_axpby<T><<<g, PW_THREADS, 0, st>>>((T)alpha, pp, (T)1, px, n3);
                }
                {
                    PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                    k_axpby<T><<<g, PW_THREADS, 0, st>>>((T)-alpha, pq, (T)1, pr, n3);
                }
                kapply(pr, pz);
                const double rzn = dot_now(pr, pz, n3);
                ++pit;
                const double res =
                    prm.space == LDDMM_SPACE_V ? std::sqrt(std::max(rzn, 0.0)) : std::sqrt(dot_now(pr, pr, n3));
                if (res <= prm.pcg_rtol * nrm0) break;
                const double beta = rzn / rz;
                {
                    PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                    k_axpby<T><<<g, PW_THREADS, 0, st>>>((T)1, pz, (T)beta, pp, n3);
                }
                rz = rzn;
            }
            R.pcg_iters[it] = pit;
            R.pcg_iters_total += pit;
            const double slope = dot_now(pg, px, n3);
            double eps = 1.0;
            bool ok = false;
            for (int t = 0; t < prm.ls_maxit; ++t) {
                {
                    PScope ps_(this, KC_MISC, 3.0 * n3 * sizeof(T));
                    k_lincomb2<T><<<g, PW_THREADS, 0, st>>>((T)1, v, (T)eps, px, pvt, n3);
                }
                const double Et = energy_at(pvt, I0, I1);
                if (status != LDDMM_OK) return status;
                if (std::isfinite(Et) && Et <= E + prm.armijo_c1 * eps * slope) {
                    ok = true;
                    break;
                }
                eps *= 0.5;
            }
            R.step[it] = ok ? eps : 0.0;
            if (!ok) {
                ls_fail = true;
                ++it;
                break;
            }
            cudaMemcpyAsync(v, pvt, n3 * sizeof(T), cudaMemcpyDeviceToDevice, st);
        }
        R.gn_iters = it;
        // final metrics: energy, relative gradient, MSE_rel, Jacobian extrema
        gradient_core(v, I0, I1, pg, LDDMM_SPACE_L2);
        if (fetch(0, prm.nt + 3) != LDDMM_OK) return status;
        R.energy[it] = hres[prm.nt + 2] + prm.weight * hres[prm.nt + 1];
        const double data = hres[prm.nt + 2];
        const T* gsp = pg;
        if (prm.space == LDDMM_SPACE_V) {
            kapply(pg, pz);
            gsp = pz;
        }
        minmax_async(gsp, n3, 60);
        if (fetch(60, 1) != LDDMM_OK) return status;
        R.gnorm_rel = g0max > 0 ? hres[60] / g0max : 0.0;
        {
            PScope ps_(this, KC_MISC, 3.0 * d.N * sizeof(T));
            k_sub<T><<<pw_grid(d.N), PW_THREADS, 0, st>>>(I0, I1, rbuf, d.N);
        }
        const double d0 = dot_now(rbuf, nullptr, d.N);
        R.mse_rel = d0 > 0 ? data / d0 : 0.0;
        T* J = rs + 9 * d.N;
        jacdet_into(u1(), J);
        minmax_async(J, d.N, 60);
        if (fetch(60, 3) != LDDMM_OK) return status;
        R.jac_max = hres[61];
        R.jac_min = hres[62];
        if (check_launch() != LDDMM_OK) return status;
        if (rep) *rep = R;
        if (!std::isfinite(R.energy[it])) return fail(LDDMM_ERR_NONFINITE);
        return ls_fail ? LDDMM_WARN_LINESEARCH : LDDMM_OK;
    }
};

EngineBase* make_engine_f64(const Dims& d, const lddmm_params& p, cudaStream_t s, lddmm_status* st);
EngineBase* make_engine_f32(const Dims& d, const lddmm_params& p, cudaStream_t s, lddmm_status* st);

}  // namespace lddmm
