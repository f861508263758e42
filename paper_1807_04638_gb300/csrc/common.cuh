// Shared device-side definitions: complex type, spectral symbols, pass jobs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lddmm {

template <class T> struct cpx;
template <> struct __align__(8) cpx<float> { float x, y; };
template <> struct __align__(16) cpx<double> { double x, y; };

template <class T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <class T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <class T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <class T> __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T> __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.x, s * a.y); }
template <class T> __device__ __forceinline__ cpx<T> cj(cpx<T> a) { return mk(a.x, -a.y); }
__device__ __forceinline__ cpx<float> ldg(const cpx<float>* p) {
    const float2 v = __ldg((const float2*)p);
    return mk(v.x, v.y);
}
__device__ __forceinline__ cpx<double> ldg(const cpx<double>* p) {
    const double2 v = __ldg((const double2*)p);
    return mk(v.x, v.y);
}
// multiply by +i (dir = +1) or -i (dir = -1)
template <class T> __device__ __forceinline__ cpx<T> rot(cpx<T> a, int dir) {
    return dir > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// Spectral symbol: scale * L_hat^lpow * (i kappa_deriv, if deriv >= 0)
// [* P, if mask], with L_hat = (1 + alpha |kappa|^2)^s, the Nyquist entry of
// i kappa zeroed and P the 2/3-rule band indicator |k_a| <= kcut_a.
struct SymD {
    double scale;
    int lpow;
    int deriv;
    int mask;
};
// The same symbol with its scale already in the compute type, as the kernels
// read it (a per-element double-to-float conversion would run on the slow
// FP64 pipe).
template <class T> struct SymT {
    T scale;
    int lpow;
    int deriv;
    int mask;
};
template <class T> inline SymT<T> to_symt(const SymD& s) {
    SymT<T> r;
    r.scale = (T)s.scale;
    r.lpow = s.lpow;
    r.deriv = s.deriv;
    r.mask = s.mask;
    return r;
}

// Per-axis symbol tables on the device (length n0, n1, n2/2+1).
template <class T> struct SpecTabs {
    const T* dk[3];   // kappa_a with the Nyquist entry zeroed (derivative symbol / i)
    const T* ksq[3];  // kappa_a^2
    T alpha;
    int s;
    int n[3];     // grid sizes (signed wave number of index k: k or k - n)
    int kcut[3];  // band of the dealiasing projector P (n when dealiasing is off)
};

// a / b for the symbols: the fast-division intrinsic in FP32 (at most two
// ulp for the positive, moderate L_hat^|lpow| values here), exact division in
// FP64
__device__ __forceinline__ float sym_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sym_div(double a, double b) { return a / b; }

template <class T>
__device__ __forceinline__ cpx<T> sym_apply(const SymT<T>& sy, const SpecTabs<T>& tb, int k0, int k1, int k2, cpx<T> v) {
    if (sy.mask) {
        // |k_a| > kcut_a  <=>  kcut_a < k_a < n_a - kcut_a (index k_a in [0, n_a))
        const bool out0 = k0 > tb.kcut[0] && k0 < tb.n[0] - tb.kcut[0];
        const bool out1 = k1 > tb.kcut[1] && k1 < tb.n[1] - tb.kcut[1];
        if (out0 || out1 || k2 > tb.kcut[2]) return mk((T)0, (T)0);
    }
    T f = sy.scale;
    if (sy.lpow != 0) {
        const T base = (T)1 + tb.alpha * (tb.ksq[0][k0] + tb.ksq[1][k1] + tb.ksq[2][k2]);
        const int e = tb.s * (sy.lpow > 0 ? sy.lpow : -sy.lpow);
        T p;
        if (e == 2) {
            p = base * base;
        } else if (e == 4) {
            p = base * base;
            p = p * p;
        } else {
            p = (T)1;
            for (int q = 0; q < e; ++q) p *= base;
        }
        f = sy.lpow > 0 ? f * p : sym_div(f, p);
    }
    if (sy.deriv >= 0) {
        int kk = sy.deriv == 0 ? k0 : (sy.deriv == 1 ? k1 : k2);
        T d = tb.dk[sy.deriv][kk] * f;
        return mk(-d * v.y, d * v.x);
    }
    return mk(f * v.x, f * v.y);
}

// The multiplier of sym_apply at one wave vector, for applying the same
// symbol to several values: (f, 0) or, with a derivative, (0, d f).
template <class T>
__device__ __forceinline__ cpx<T> sym_coef(const SymT<T>& sy, const SpecTabs<T>& tb, int k0, int k1, int k2) {
    return sym_apply(sy, tb, k0, k1, k2, mk((T)1, (T)0));
}
// v times such a multiplier (one of its parts is zero)
template <class T> __device__ __forceinline__ cpx<T> sym_mul(cpx<T> s, cpx<T> v) {
    return mk(s.x * v.x - s.y * v.y, s.x * v.y + s.y * v.x);
}

// One FFT axis: length, radix plan, twiddle table e^{-2 pi i t / n}, t < n.
struct FFTAxis {
    int n;
    int nst;
    int rad[12];
    const void* tw;
};

constexpr int MAXI = 4;   // inputs per job
constexpr int MAXO = 4;   // outputs per job
constexpr int MAXB = 4;   // un-transformed bases per job
constexpr int MAXJOBS = 24;

// One transform job inside a pass.
//  inverse direction: x = sum_i isym[i].scale * in[i];  out[o] = IFFT(osym[o] . x)
//  forward direction: out[0] = sum_b bcoef[b] * base[b] + sum_i isym[i] . FFT(in[i])
struct PassJob {
    const void* in[MAXI];
    SymD isym[MAXI];
    void* out[MAXO];
    SymD osym[MAXO];
    const void* base[MAXB];
    double bcoef[MAXB];
    int nin, nout, nb, pad_;
};
// A job as the kernels read it: scalars in the compute type.
template <class T> struct PassJobT {
    const void* in[MAXI];
    SymT<T> isym[MAXI];
    void* out[MAXO];
    SymT<T> osym[MAXO];
    const void* base[MAXB];
    T bcoef[MAXB];
    int nin, nout, nb, pad_;
};
template <class T> inline PassJobT<T> to_jobt(const PassJob& j) {
    PassJobT<T> r;
    for (int i = 0; i < MAXI; ++i) {
        r.in[i] = j.in[i];
        r.isym[i] = to_symt<T>(j.isym[i]);
    }
    for (int i = 0; i < MAXO; ++i) {
        r.out[i] = j.out[i];
        r.osym[i] = to_symt<T>(j.osym[i]);
    }
    for (int i = 0; i < MAXB; ++i) {
        r.base[i] = j.base[i];
        r.bcoef[i] = (T)j.bcoef[i];
    }
    r.nin = j.nin;
    r.nout = j.nout;
    r.nb = j.nb;
    r.pad_ = 0;
    return r;
}

// Division by a divisor d (1 <= d < 2^24) fixed for a launch, for numerators
// n < 2^24, by one 32 x 32 -> 64-bit multiply and a shift: with
// l = ceil(log2 d), sh = 24 + l and m = ceil(2^sh / d) (m < 2^26), n / d =
// (n m) >> sh exactly, since 2^sh <= m d <= 2^sh + 2^l (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// Thm. 4.2).  Built on the host; the kernels only multiply.
struct FastDiv {
    unsigned d, m;
    int sh;
    FastDiv() : d(1), m(1u << 24), sh(24) {}
    explicit FastDiv(unsigned dd) : d(dd) {
        int l = 0;
        while ((1u << l) < dd) ++l;
        sh = 24 + l;
        m = (unsigned)(((1ull << sh) + dd - 1) / dd);
    }
    __device__ __forceinline__ unsigned div(unsigned n) const {
        return (unsigned)(((unsigned long long)n * m) >> sh);
    }
};

template <class T> struct PassParams {
    FFTAxis ax;
    int n0, n1, n2, n2h;
    int TL, P, Ph;     // lines per tile, line pitch, half-spectrum pitch (axis-2 pass)
    int sign;          // -1 forward, +1 inverse
    // Band of the transform (register-blocked passes): only the k2 planes
    // k2 < nb2 and the k1 columns [0, c1) U [s1, n1) are transformed; every
    // other spectral entry is treated as zero on input and left unwritten on
    // output.  The full transform has nb2 = n2h, c1 = s1 = n1.
    int nb2, c1, s1;
    // register-blocked C2C passes: divisions by the launch's tile count, by
    // the tiles per k2 plane (axis 0) and by n0 (axis 1)
    FastDiv fd_tiles, fd_tpk, fd_n0;
    SpecTabs<T> tabs;
    int njobs;
    PassJobT<T> jobs[MAXJOBS];
};
template <class T> inline void full_band(PassParams<T>& p) {
    p.nb2 = p.n2h;
    p.c1 = p.n1;
    p.s1 = p.n1;
}

}  // namespace lddmm
