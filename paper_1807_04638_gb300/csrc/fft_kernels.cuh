// Shared-memory Stockham FFT passes over 3D periodic fields.
//
// Spectral layout [k2][k0][k1] (k1 fastest), real layout [i0][i1][i2].
// A 3D real transform is three passes:
//   axis 2 (R2C / C2R, two real rows packed into one complex line, written /
//   read transposed into the [k2][row] spectral layout, row = i0*n1 + i1),
//   axis 1 (C2C on contiguous lines of n1), axis 0 (C2C on lines strided by n1).
// Each pass also applies spectral symbols (derivatives, powers of L), fans one
// input out into several outputs (inverse direction) or combines several
// inputs and un-transformed bases into one output (forward direction).
#pragma once
#include "common.cuh"

namespace lddmm {

constexpr int FFT_THREADS = 256;

// ---------------------------------------------------------------- butterflies
template <class T> struct Rad {
    static __device__ __forceinline__ void r2(cpx<T>* v) {
        cpx<T> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
    // dir = sign of the exponent (-1 forward, +1 inverse)
    static __device__ __forceinline__ void r4(cpx<T>* v, int dir) {
        cpx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = rot(v[1] - v[3], dir);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    }
    static __device__ __forceinline__ void r3(cpx<T>* v, int dir) {
        const T h = (T)0.86602540378443864676;  // sqrt(3)/2
        cpx<T> s = v[1] + v[2], d = v[1] - v[2];
        cpx<T> m = v[0] - (T)0.5 * s;
        cpx<T> q = rot((T)h * d, dir);
        v[0] = v[0] + s;
        v[1] = m + q;
        v[2] = m - q;
    }
    static __device__ __forceinline__ void r5(cpx<T>* v, int dir) {
        const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
        const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
        cpx<T> a1 = v[1] + v[4], b1 = v[1] - v[4], a2 = v[2] + v[3], b2 = v[2] - v[3];
        cpx<T> x0 = v[0];
        cpx<T> p1 = x0 + c1 * a1 + c2 * a2;
        cpx<T> p2 = x0 + c2 * a1 + c1 * a2;
        cpx<T> q1 = rot(s1 * b1 + s2 * b2, dir);
        cpx<T> q2 = rot(s2 * b1 - s1 * b2, dir);
        v[0] = x0 + a1 + a2;
        v[1] = p1 + q1;
        v[4] = p1 - q1;
        v[2] = p2 + q2;
        v[3] = p2 - q2;
    }
};

// In-tile Stockham transform of `ncols` lines of length n stored at
// src[c*P + i].  Ping-pongs between src and dst; returns the buffer holding
// the result.  All threads of the block must call it.
template <class T>
__device__ cpx<T>* fft_tile(cpx<T>* src, cpx<T>* dst, int ncols, int P, const FFTAxis& ax, int dir) {
    const int n = ax.n;
    const cpx<T>* tw = (const cpx<T>*)ax.tw;
    int Ns = 1;
    for (int st = 0; st < ax.nst; ++st) {
        const int R = ax.rad[st];
        const int m = n / R;
        const int twstep = n / (Ns * R);
        const int items = ncols * m;
        for (int w = threadIdx.x; w < items; w += blockDim.x) {
            const int c = w % ncols, j = w / ncols;
            const int k = j % Ns;
            cpx<T> v[5];
            const cpx<T>* s = src + c * P + j;
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                if (r < R) {
                    cpx<T> x = s[r * m];
                    if (r > 0 && k > 0) {
                        cpx<T> t = ldg(&tw[k * r * twstep]);
                        if (dir > 0) t.y = -t.y;
                        x = x * t;
                    }
                    v[r] = x;
                }
            }
            if (R == 4) Rad<T>::r4(v, dir);
            else if (R == 2) Rad<T>::r2(v);
            else if (R == 3) Rad<T>::r3(v, dir);
            else Rad<T>::r5(v, dir);
            cpx<T>* d = dst + c * P + (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) d[r * Ns] = v[r];
        }
        __syncthreads();
        cpx<T>* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// ---------------------------------------------------------------- C2C passes
// AXIS 1: lines along k1 (contiguous, line id = k2*n0 + k0).
// AXIS 0: lines along k0 (stride n1) for a tile of TL consecutive k1.
template <class T, int AXIS>
__global__ void __launch_bounds__(FFT_THREADS) k_pass_c2c(const __grid_constant__ PassParams<T> pp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TL = pp.TL, P = pp.P, n = pp.ax.n;
    cpx<T>* X = (cpx<T>*)smem_raw;
    cpx<T>* A = X + TL * P;
    cpx<T>* B = A + TL * P;
    const PassJobT<T>& job = pp.jobs[blockIdx.y];
    const int n0 = pp.n0, n1 = pp.n1, n2h = pp.n2h;

    int ncols, line0 = 0, k2t = 0, k10 = 0;
    if (AXIS == 1) {
        const int lines = n2h * n0;
        line0 = blockIdx.x * TL;
        ncols = min(TL, lines - line0);
    } else {
        const int tpk = (n1 + TL - 1) / TL;
        k2t = blockIdx.x / tpk;
        k10 = (blockIdx.x % tpk) * TL;
        ncols = min(TL, n1 - k10);
    }
    const int total = ncols * n;
    // element e -> (c, i), global offset, frequency indices
    auto geo = [&](int e, int& c, int& i, size_t& g, int& k0, int& k1, int& k2) {
        if (AXIS == 1) {
            c = e / n;
            i = e % n;
            const int line = line0 + c;
            g = (size_t)line * n1 + i;
            k2 = line / n0;
            k0 = line % n0;
            k1 = i;
        } else {
            c = e % ncols;
            i = e / ncols;
            g = ((size_t)k2t * n0 + i) * n1 + k10 + c;
            k0 = i;
            k1 = k10 + c;
            k2 = k2t;
        }
    };

    if (pp.sign > 0) {
        // ---- inverse: lincomb load, per-output symbol, IFFT, store
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int c, i, k0, k1, k2;
            size_t g;
            geo(e, c, i, g, k0, k1, k2);
            cpx<T> acc = mk((T)0, (T)0);
            for (int b = 0; b < job.nin; ++b) {
                cpx<T> v = ((const cpx<T>*)job.in[b])[g];
                acc = acc + job.isym[b].scale * v;
            }
            X[c * P + i] = acc;
        }
        __syncthreads();
        for (int o = 0; o < job.nout; ++o) {
            const SymT<T> sy = job.osym[o];
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                int c, i, k0, k1, k2;
                size_t g;
                geo(e, c, i, g, k0, k1, k2);
                A[c * P + i] = sym_apply(sy, pp.tabs, k0, k1, k2, X[c * P + i]);
            }
            __syncthreads();
            cpx<T>* R = fft_tile(A, B, ncols, P, pp.ax, +1);
            cpx<T>* out = (cpx<T>*)job.out[o];
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                int c, i, k0, k1, k2;
                size_t g;
                geo(e, c, i, g, k0, k1, k2);
                out[g] = R[c * P + i];
            }
            __syncthreads();
        }
    } else {
        // ---- forward: FFT each input, post-symbol, accumulate, add bases, store
        for (int q = 0; q < job.nin; ++q) {
            const cpx<T>* in = (const cpx<T>*)job.in[q];
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                int c, i, k0, k1, k2;
                size_t g;
                geo(e, c, i, g, k0, k1, k2);
                A[c * P + i] = in[g];
            }
            __syncthreads();
            cpx<T>* R = fft_tile(A, B, ncols, P, pp.ax, -1);
            const SymT<T> sy = job.isym[q];
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                int c, i, k0, k1, k2;
                size_t g;
                geo(e, c, i, g, k0, k1, k2);
                cpx<T> v = sym_apply(sy, pp.tabs, k0, k1, k2, R[c * P + i]);
                X[c * P + i] = q == 0 ? v : X[c * P + i] + v;
            }
            __syncthreads();
        }
        cpx<T>* out = (cpx<T>*)job.out[0];
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int c, i, k0, k1, k2;
            size_t g;
            geo(e, c, i, g, k0, k1, k2);
            cpx<T> v = X[c * P + i];
            for (int b = 0; b < job.nb; ++b) v = v + job.bcoef[b] * ((const cpx<T>*)job.base[b])[g];
            out[g] = v;
        }
    }
}

// ---------------------------------------------------------------- axis-2 pass
// Rows r = i0*n1 + i1 in [0, n0*n1); a block owns 2*TL consecutive rows packed
// as TL complex lines z = row(2c) + i row(2c+1).  The half spectrum of the
// block is staged in H[row][k2] (pitch Ph); spectral layout [k2][row].
template <class T>
__global__ void __launch_bounds__(FFT_THREADS) k_pass_axis2(const __grid_constant__ PassParams<T> pp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TL = pp.TL, P = pp.P, Ph = pp.Ph, n2 = pp.n2, n2h = pp.n2h;
    const int rows = pp.n0 * pp.n1;
    cpx<T>* H = (cpx<T>*)smem_raw;
    cpx<T>* A = H + 2 * TL * Ph;
    cpx<T>* B = A + TL * P;
    const PassJobT<T>& job = pp.jobs[blockIdx.y];
    const int r0 = blockIdx.x * 2 * TL;
    const int nr = min(2 * TL, rows - r0);
    const int npair = (nr + 1) / 2;
    const bool even = (n2 % 2) == 0;

    if (pp.sign > 0) {
        // ---- C2R: load half spectra (lincomb), per output symbol, pack, IFFT, store rows
        for (int e = threadIdx.x; e < 2 * TL * n2h; e += blockDim.x) {
            const int row = e % (2 * TL), k = e / (2 * TL);
            cpx<T> acc = mk((T)0, (T)0);
            if (row < nr)
                for (int b = 0; b < job.nin; ++b)
                    acc = acc + job.isym[b].scale * ((const cpx<T>*)job.in[b])[(size_t)k * rows + r0 + row];
            H[row * Ph + k] = acc;
        }
        __syncthreads();
        for (int o = 0; o < job.nout; ++o) {
            const SymT<T> sy = job.osym[o];
            for (int e = threadIdx.x; e < npair * n2; e += blockDim.x) {
                const int c = e / n2, k = e % n2;
                const bool lo = k < n2h;
                const int kk = lo ? k : n2 - k;
                cpx<T> a = sym_apply(sy, pp.tabs, 0, 0, kk, H[(2 * c) * Ph + kk]);
                cpx<T> b = sym_apply(sy, pp.tabs, 0, 0, kk, H[(2 * c + 1) * Ph + kk]);
                if (kk == 0 || (even && kk == n2 / 2)) {
                    a.y = 0;
                    b.y = 0;
                }
                if (!lo) {
                    a = cj(a);
                    b = cj(b);
                }
                A[c * P + k] = mk(a.x - b.y, a.y + b.x);
            }
            __syncthreads();
            cpx<T>* R = fft_tile(A, B, npair, P, pp.ax, +1);
            T* out = (T*)job.out[o];
            for (int e = threadIdx.x; e < npair * n2; e += blockDim.x) {
                const int c = e / n2, i = e % n2;
                const cpx<T> z = R[c * P + i];
                out[(size_t)(r0 + 2 * c) * n2 + i] = z.x;
                if (2 * c + 1 < nr) out[(size_t)(r0 + 2 * c + 1) * n2 + i] = z.y;
            }
            __syncthreads();
        }
    } else {
        // ---- R2C: for each real input, pack rows, FFT, split, post-symbol, accumulate in H
        for (int q = 0; q < job.nin; ++q) {
            const T* in = (const T*)job.in[q];
            for (int e = threadIdx.x; e < npair * n2; e += blockDim.x) {
                const int c = e / n2, i = e % n2;
                const T a = in[(size_t)(r0 + 2 * c) * n2 + i];
                const T b = (2 * c + 1 < nr) ? in[(size_t)(r0 + 2 * c + 1) * n2 + i] : (T)0;
                A[c * P + i] = mk(a, b);
            }
            __syncthreads();
            cpx<T>* R = fft_tile(A, B, npair, P, pp.ax, -1);
            const SymT<T> sy = job.isym[q];
            for (int e = threadIdx.x; e < npair * n2h; e += blockDim.x) {
                const int c = e / n2h, k = e % n2h;
                const cpx<T> zk = R[c * P + k];
                const cpx<T> zn = cj(R[c * P + (k == 0 ? 0 : n2 - k)]);
                const cpx<T> fa = (T)0.5 * (zk + zn);
                const cpx<T> fb = rot((T)0.5 * (zk - zn), -1);
                const cpx<T> sa = sym_apply(sy, pp.tabs, 0, 0, k, fa);
                const cpx<T> sb = sym_apply(sy, pp.tabs, 0, 0, k, fb);
                cpx<T>* ha = &H[(2 * c) * Ph + k];
                cpx<T>* hb = &H[(2 * c + 1) * Ph + k];
                *ha = q == 0 ? sa : *ha + sa;
                *hb = q == 0 ? sb : *hb + sb;
            }
            __syncthreads();
        }
        cpx<T>* out = (cpx<T>*)job.out[0];
        for (int e = threadIdx.x; e < 2 * TL * n2h; e += blockDim.x) {
            const int row = e % (2 * TL), k = e / (2 * TL);
            if (row < nr) out[(size_t)k * rows + r0 + row] = H[row * Ph + k];
        }
    }
}

}  // namespace lddmm
