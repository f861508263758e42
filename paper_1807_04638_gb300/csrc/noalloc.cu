// Metric operator L^power without any device allocation.
//
// Some callers cannot allocate device memory: code that runs while a CUDA
// graph is being captured, real-time loops that must not enter the
// allocator, and plug-ins whose host application owns every device
// allocation.  They cannot create an lddmm_handle (which cudaMallocs its
// workspace), so this entry point takes its scratch from a fixed array that
// lives in the library's device image instead.
//
// The scratch is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES; every
// GPU that loads the library holds it until the process exits.  In host code
// the array's name is only a host-side stand-in for the symbol, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.  That lookup happens in the
// first call on each device; make that first call before any stream capture.
// All calls share the one array and it keeps the last call's contents: every
// call rewrites the tables and buffers it reads, and calls that overlap on
// the GPU (on different streams, or from different host threads without
// ordering) race on it.
#include <mutex>

#include "engine.cuh"

namespace lddmm {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)24 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Radices 4, 2, 3, 5 (same order as the handle's plans), without a heap.
static int noalloc_radix_plan(int n, int* rad) {
    int k = 0, m = n;
    const int rs[4] = {4, 2, 3, 5};
    for (int q = 0; q < 4; ++q)
        while (m % rs[q] == 0 && k < 12) {
            rad[k++] = rs[q];
            m /= rs[q];
        }
    return k;
}

// Twiddles e^{-2 pi i t / n_a} and the symbol tables, written into scratch.
template <class T>
__global__ void k_noalloc_tables(int n0, int n1, int n2, double l0, double l1, double l2, cpx<T>* tw0, cpx<T>* tw1,
                                 cpx<T>* tw2, T* dk0, T* dk1, T* dk2, T* ks0, T* ks1, T* ks2) {
    const int ns[3] = {n0, n1, n2};
    const double ls[3] = {l0, l1, l2};
    cpx<T>* tws[3] = {tw0, tw1, tw2};
    T* dks[3] = {dk0, dk1, dk2};
    T* kss[3] = {ks0, ks1, ks2};
    for (int a = 0; a < 3; ++a) {
        const int n = ns[a];
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
            double sn, cs;
            sincospi(-2.0 * (double)t / (double)n, &sn, &cs);
            tws[a][t] = mk((T)cs, (T)sn);
            const int nk = a < 2 ? n : n / 2 + 1;
            if (t < nk) {
                const int sk = (a < 2 && t >= (n + 1) / 2) ? t - n : t;
                const double kap = 2.0 * 3.14159265358979323846 / ls[a] * (double)sk;
                kss[a][t] = (T)(kap * kap);
                dks[a][t] = ((n % 2 == 0) && t == n / 2) ? (T)0 : (T)kap;
            }
        }
    }
}

template <class T>
static lddmm_status noalloc_run(const Dims& d, double alpha, int s, int power, const T* in, T* out, int ncomp,
                                cudaStream_t st) {
    using C = cpx<T>;
    void* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return LDDMM_ERR_CUDA;
    // carve the scratch
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        unsigned char* p = (unsigned char*)base + off;
        off += bytes;
        return (void*)p;
    };
    const int ns[3] = {d.n0, d.n1, d.n2};
    const int nk[3] = {d.n0, d.n1, d.n2h};
    C* tw[3];
    T *dk[3], *ks[3];
    for (int a = 0; a < 3; ++a) tw[a] = (C*)carve(ns[a] * sizeof(C));
    for (int a = 0; a < 3; ++a) dk[a] = (T*)carve(nk[a] * sizeof(T));
    for (int a = 0; a < 3; ++a) ks[a] = (T*)carve(nk[a] * sizeof(T));
    C* A = (C*)carve(d.NS * sizeof(C));
    C* B = (C*)carve(d.NS * sizeof(C));
    if (off > NOALLOC_SCRATCH_BYTES) return LDDMM_ERR_TOO_LARGE;

    k_noalloc_tables<T><<<4, 128, 0, st>>>(d.n0, d.n1, d.n2, d.len[0], d.len[1], d.len[2], tw[0], tw[1], tw[2], dk[0],
                                          dk[1], dk[2], ks[0], ks[1], ks[2]);
    SpecTabs<T> tabs;
    for (int a = 0; a < 3; ++a) {
        tabs.dk[a] = dk[a];
        tabs.ksq[a] = ks[a];
        tabs.n[a] = ns[a];
        tabs.kcut[a] = ns[a];
    }
    tabs.alpha = (T)alpha;
    tabs.s = s;

    // generic-pass tile geometry (as the handle uses it)
    const size_t budget = 150 * 1024;
    int TLc[2], Pc[2];
    size_t smc[2];
    for (int a = 0; a < 2; ++a) {
        Pc[a] = (ns[a] % 2 == 0) ? ns[a] + 1 : ns[a];
        TLc[a] = 16;
        while (TLc[a] > 1 && (size_t)3 * TLc[a] * Pc[a] * sizeof(C) > budget) TLc[a] /= 2;
        smc[a] = (size_t)3 * TLc[a] * Pc[a] * sizeof(C);
    }
    const int P2 = (d.n2 % 2 == 0) ? d.n2 + 1 : d.n2;
    const int Ph2 = (d.n2h % 2 == 0) ? d.n2h + 1 : d.n2h;
    int TL2 = 16;
    while (TL2 > 1 && ((size_t)2 * TL2 * Ph2 + 2 * TL2 * P2) * sizeof(C) > budget) TL2 /= 2;
    const size_t sm2 = ((size_t)2 * TL2 * Ph2 + 2 * TL2 * P2) * sizeof(C);
    bool fast[3];
    for (int a = 0; a < 3; ++a) {
        PassParams<T> dummy;
        const bool aligned = a != 0 || sizeof(T) == 8 || ns[1] % 2 == 0;
        fast[a] = FastPass<T>::has(ns[a]) && aligned && !force_generic_fft() &&
                  FastPass<T>::launch(ns[a], a, 0, dummy, 0, 0, 0, 0, 0, st, true);
    }
    if (!raise_smem_limit(k_pass_c2c<T, 0>, smc[0]) || !raise_smem_limit(k_pass_c2c<T, 1>, smc[1]) ||
        !raise_smem_limit(k_pass_axis2<T>, sm2))
        return LDDMM_ERR_CUDA;

    auto one = [&](int axis, int sign, const void* src, void* dst, SymD sy) {
        PassParams<T> pp;
        memset(&pp, 0, sizeof(pp));
        pp.ax.n = ns[axis];
        pp.ax.nst = noalloc_radix_plan(ns[axis], pp.ax.rad);
        pp.ax.tw = tw[axis];
        pp.n0 = d.n0;
        pp.n1 = d.n1;
        pp.n2 = d.n2;
        pp.n2h = d.n2h;
        pp.sign = sign;
        full_band(pp);
        pp.tabs = tabs;
        pp.njobs = 1;
        PassJobT<T>& j = pp.jobs[0];
        j.nin = 1;
        j.in[0] = src;
        j.nout = 1;
        j.out[0] = dst;
        SymT<T> unit;
        unit.scale = (T)1;
        unit.lpow = 0;
        unit.deriv = -1;
        unit.mask = 0;
        const SymT<T> syt = to_symt<T>(sy);
        j.isym[0] = sign > 0 ? unit : syt;
        j.osym[0] = sign > 0 ? syt : unit;
        if (fast[axis]) {
            FastPass<T>::launch(ns[axis], axis, sign, pp, 1, d.rows, d.n0, d.n1, d.n2h, st);
        } else if (axis == 2) {
            pp.TL = TL2;
            pp.P = P2;
            pp.Ph = Ph2;
            const int gx = (int)((d.rows + 2 * TL2 - 1) / (2 * TL2));
            k_pass_axis2<T><<<dim3(gx, 1), FFT_THREADS, sm2, st>>>(pp);
        } else if (axis == 1) {
            pp.TL = TLc[1];
            pp.P = Pc[1];
            const int gx = (int)(((size_t)d.n2h * d.n0 + TLc[1] - 1) / TLc[1]);
            k_pass_c2c<T, 1><<<dim3(gx, 1), FFT_THREADS, smc[1], st>>>(pp);
        } else {
            pp.TL = TLc[0];
            pp.P = Pc[0];
            const int gx = d.n2h * ((d.n1 + TLc[0] - 1) / TLc[0]);
            k_pass_c2c<T, 0><<<dim3(gx, 1), FFT_THREADS, smc[0], st>>>(pp);
        }
    };
    SymD unit;
    unit.scale = 1.0;
    unit.lpow = 0;
    unit.deriv = -1;
    unit.mask = 0;
    SymD lp = unit;
    lp.lpow = power;
    SymD inv = unit;
    inv.scale = 1.0 / (double)d.N;
    for (int c = 0; c < ncomp; ++c) {
        const T* x = in + (size_t)c * d.N;
        T* y = out + (size_t)c * d.N;
        one(2, -1, x, A, unit);  // rows -> [k2][row]
        one(1, -1, A, B, unit);
        one(0, -1, B, A, lp);    // full spectrum times L_hat^power
        one(0, +1, A, B, inv);   // 1/N normalisation of the inverse
        one(1, +1, B, A, unit);
        one(2, +1, A, y, unit);
    }
    return cudaGetLastError() == cudaSuccess ? LDDMM_OK : LDDMM_ERR_CUDA;
}

}  // namespace lddmm

using namespace lddmm;

extern "C" lddmm_status lddmm_apply_metric_noalloc(const lddmm_grid* g, double alpha, int s, int power, int dtype,
                                                   const void* in, void* out, int ncomp, void* cuda_stream) {
    Dims d;
    if (!make_dims(g, &d)) return LDDMM_ERR_SHAPE;
    if (!in || !out || ncomp < 1 || !(alpha > 0) || s < 1 || s > 8 || power < -4 || power > 4) return LDDMM_ERR_ARG;
    if (dtype != LDDMM_F64 && dtype != LDDMM_F32) return LDDMM_ERR_ARG;
    if (lddmm_apply_metric_noalloc_scratch_bytes(g, dtype) > NOALLOC_SCRATCH_BYTES) return LDDMM_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return dtype == LDDMM_F64 ? noalloc_run<double>(d, alpha, s, power, (const double*)in, (double*)out, ncomp, st)
                              : noalloc_run<float>(d, alpha, s, power, (const float*)in, (float*)out, ncomp, st);
}

extern "C" size_t lddmm_apply_metric_noalloc_scratch_bytes(const lddmm_grid* g, int dtype) {
    Dims d;
    if (!make_dims(g, &d)) return 0;
    const size_t t = dtype == LDDMM_F64 ? 8 : 4;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t b = 0;
    const int ns[3] = {d.n0, d.n1, d.n2};
    const int nk[3] = {d.n0, d.n1, d.n2h};
    for (int a = 0; a < 3; ++a) b += al(ns[a] * 2 * t);
    for (int a = 0; a < 3; ++a) b += 2 * al(nk[a] * t);
    b += 2 * al(d.NS * 2 * t);
    return b;
}

extern "C" size_t lddmm_apply_metric_noalloc_capacity(void) { return NOALLOC_SCRATCH_BYTES; }
