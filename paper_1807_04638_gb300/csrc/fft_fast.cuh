// Register-blocked FFT passes for line lengths known at compile time.
//
// Each thread owns E = N / TPL elements of one line, at positions t + TPL*m
// (t = thread index within the line, m = 0..E-1).  A Stockham stage of radix
// R reads, for butterfly b (j = t + TPL*b), the elements j + r*N/R, which are
// exactly the thread's own registers b + (E/R)*r; so every stage starts from
// registers, computes its butterflies there, and only the scattered writes of
// a non-final stage go through shared memory (ping-pong tiles, one barrier per
// exchange).  The final stage leaves element t + TPL*m in register m, which
// is stored straight to global memory.  Same jobs and layouts as the generic
// passes in fft_kernels.cuh.
#pragma once
#include "common.cuh"
#include "fft_kernels.cuh"

namespace lddmm {

// Radix plans packed one radix per nibble, stage 0 in the low nibble.
template <int N> struct FastPlan { static constexpr bool ok = false; };
template <> struct FastPlan<32> { static constexpr bool ok = true; static constexpr int E = 8, RADS = 0x48; };
template <> struct FastPlan<64> { static constexpr bool ok = true; static constexpr int E = 8, RADS = 0x88; };
template <> struct FastPlan<128> { static constexpr bool ok = true; static constexpr int E = 8, RADS = 0x448; };
template <> struct FastPlan<256> { static constexpr bool ok = true; static constexpr int E = 8, RADS = 0x488; };

constexpr int FAST_THREADS = 256;
// Resident blocks per SM the register budget is sized for: 4 for FP32
// (<= 64 registers), 2 for FP64, so that enough loads are in flight to hide
// DRAM latency.
template <class T> struct FastOcc { static constexpr int value = sizeof(T) == 4 ? 4 : 2; };

template <class T> struct Rad8 {
    // y_k = sum_r x_r w^{rk}, w = e^{dir 2 pi i / 8}
    static __device__ __forceinline__ void run(cpx<T>* v, int dir) {
        const T h = (T)0.70710678118654752440;
        cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
        cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
        Rad<T>::r4(e, dir);
        Rad<T>::r4(o, dir);
        // twiddles w^k, k = 0..3
        const cpx<T> o1 = mk(h * (o[1].x - dir * o[1].y), h * (o[1].y + dir * o[1].x));  // o1 * (1 + dir i)/sqrt2
        const cpx<T> o2 = rot(o[2], dir);
        const cpx<T> o3 = mk(h * (-o[3].x - dir * o[3].y), h * (-o[3].y + dir * o[3].x));  // o3 * (-1 + dir i)/sqrt2
        v[0] = e[0] + o[0];
        v[4] = e[0] - o[0];
        v[1] = e[1] + o1;
        v[5] = e[1] - o1;
        v[2] = e[2] + o2;
        v[6] = e[2] - o2;
        v[3] = e[3] + o3;
        v[7] = e[3] - o3;
    }
};

template <class T, int R>
__device__ __forceinline__ void dft_r(cpx<T>* v, int dir) {
    if constexpr (R == 2) Rad<T>::r2(v);
    else if constexpr (R == 4) Rad<T>::r4(v, dir);
    else if constexpr (R == 8) Rad8<T>::run(v, dir);
    else if constexpr (R == 3) Rad<T>::r3(v, dir);
    else Rad<T>::r5(v, dir);
}

// Shared-memory index of element p of line c.
//  MAP 1 (t fastest in a warp): one pad slot every 8 elements inside a line.
//  MAP 0 (c fastest in a warp): odd line pitch.
template <int N, int MAP> struct SIdx {
    static constexpr int LP = MAP == 1 ? N + N / 8 + 1 : N + 1;
    static __device__ __forceinline__ int at(int c, int p) { return MAP == 1 ? c * LP + p + (p >> 3) : c * LP + p; }
};

template <class T, int N, int E, int TPL, int RADS, int S, int NS, int MAP>
__device__ __forceinline__ void fast_stages(cpx<T> (&x)[E], cpx<T>* b0, cpx<T>* b1, int c, int t, const cpx<T>* tw,
                                            int dir) {
    constexpr int R = (RADS >> (4 * S)) & 0xF;
    constexpr bool LAST = NS * R == N;
    constexpr int B = E / R;
    static_assert(B * R == E, "radix must divide the per-thread element count");
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + TPL * b;
        const int k = j % NS;
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cpx<T> a = x[b + B * r];
            if (NS > 1 && r > 0) {
                cpx<T> w = ldg(&tw[k * r * (N / (NS * R))]);
                if (dir > 0) w.y = -w.y;
                a = a * w;
            }
            v[r] = a;
        }
        dft_r<T, R>(v, dir);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[b + B * r] = v[r];
        } else {
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) b0[SIdx<N, MAP>::at(c, base + r * NS)] = v[r];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) x[m] = b0[SIdx<N, MAP>::at(c, t + TPL * m)];
        fast_stages<T, N, E, TPL, RADS, S + 1, NS * R, MAP>(x, b1, b0, c, t, tw, dir);
    }
}

template <class T, int N, int MAP>
__device__ __forceinline__ void fast_fft(cpx<T> (&x)[FastPlan<N>::E], cpx<T>* b0, cpx<T>* b1, int c, int t,
                                         const cpx<T>* tw, int dir) {
    constexpr int E = FastPlan<N>::E;
    __syncthreads();  // the tiles may still be read by the previous transform
    fast_stages<T, N, E, N / E, FastPlan<N>::RADS, 0, 1, MAP>(x, b0, b1, c, t, tw, dir);
}

// ---------------------------------------------------------------- C2C passes
// AXIS 1: lines along k1 (contiguous), MAP 1: a warp covers 32/TPL lines.
// AXIS 0: lines along k0 (stride n1), MAP 0: a warp covers TL columns.
template <class T, int N, int AXIS>
__global__ void __launch_bounds__(FAST_THREADS, FastOcc<T>::value) k_fast_c2c(const __grid_constant__ PassParams<T> pp) {
    constexpr int E = FastPlan<N>::E;
    constexpr int TPL = N / E;
    constexpr int TL = FAST_THREADS / TPL;
    constexpr int MAP = AXIS == 1 ? 1 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* b0 = (cpx<T>*)smem_raw;
    cpx<T>* b1 = b0 + TL * SIdx<N, MAP>::LP;
    const PassJob& job = pp.jobs[blockIdx.y];
    const cpx<T>* tw = (const cpx<T>*)pp.ax.tw;
    const int n0 = pp.n0, n1 = pp.n1, n2h = pp.n2h;
    int c, t;
    if (MAP == 1) {
        c = threadIdx.x / TPL;
        t = threadIdx.x % TPL;
    } else {
        c = threadIdx.x % TL;
        t = threadIdx.x / TL;
    }
    size_t gbase;
    size_t gstride;
    int k0b = 0, k1b = 0, k2b = 0;
    bool valid;
    if (AXIS == 1) {
        const int line = blockIdx.x * TL + c;
        valid = line < n2h * n0;
        const int l = valid ? line : 0;
        gbase = (size_t)l * n1;
        gstride = 1;
        k2b = l / n0;
        k0b = l % n0;
    } else {
        const int tpk = (n1 + TL - 1) / TL;
        const int k2t = blockIdx.x / tpk;
        const int k1 = (blockIdx.x % tpk) * TL + c;
        valid = k1 < n1;
        gbase = (size_t)k2t * n0 * n1 + (valid ? k1 : 0);
        gstride = n1;
        k1b = valid ? k1 : 0;
        k2b = k2t;
    }
    auto freq = [&](int p, int& k0, int& k1, int& k2) {
        k0 = AXIS == 0 ? p : k0b;
        k1 = AXIS == 1 ? p : k1b;
        k2 = k2b;
    };
    cpx<T> x[E];
    if (pp.sign > 0) {
        cpx<T> xin[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const size_t g = gbase + (size_t)(t + TPL * m) * gstride;
            cpx<T> acc = mk((T)0, (T)0);
            if (valid)
                for (int b = 0; b < job.nin; ++b) acc = acc + (T)job.isym[b].scale * ((const cpx<T>*)job.in[b])[g];
            xin[m] = acc;
        }
        for (int o = 0; o < job.nout; ++o) {
            const SymD sy = job.osym[o];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                int k0, k1, k2;
                freq(t + TPL * m, k0, k1, k2);
                x[m] = sym_apply(sy, pp.tabs, k0, k1, k2, xin[m]);
            }
            fast_fft<T, N, MAP>(x, b0, b1, c, t, tw, +1);
            if (valid) {
                cpx<T>* out = (cpx<T>*)job.out[o];
#pragma unroll
                for (int m = 0; m < E; ++m) out[gbase + (size_t)(t + TPL * m) * gstride] = x[m];
            }
        }
    } else {
        cpx<T> acc[E];
#pragma unroll
        for (int m = 0; m < E; ++m) acc[m] = mk((T)0, (T)0);
        for (int q = 0; q < job.nin; ++q) {
            const cpx<T>* in = (const cpx<T>*)job.in[q];
#pragma unroll
            for (int m = 0; m < E; ++m)
                x[m] = valid ? in[gbase + (size_t)(t + TPL * m) * gstride] : mk((T)0, (T)0);
            fast_fft<T, N, MAP>(x, b0, b1, c, t, tw, -1);
            const SymD sy = job.isym[q];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                int k0, k1, k2;
                freq(t + TPL * m, k0, k1, k2);
                acc[m] = acc[m] + sym_apply(sy, pp.tabs, k0, k1, k2, x[m]);
            }
        }
        if (valid) {
            cpx<T>* out = (cpx<T>*)job.out[0];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const size_t g = gbase + (size_t)(t + TPL * m) * gstride;
                cpx<T> v = acc[m];
                for (int b = 0; b < job.nb; ++b) v = v + (T)job.bcoef[b] * ((const cpx<T>*)job.base[b])[g];
                out[g] = v;
            }
        }
    }
}

// ---------------------------------------------------------------- axis-2 pass
// A block owns 2*TL consecutive rows, packed as TL complex lines; the half
// spectrum of the block is staged in H[row][k] (pitch Ph) for the transposed
// [k2][row] spectral layout.
template <class T, int N>
__global__ void __launch_bounds__(FAST_THREADS, FastOcc<T>::value) k_fast_axis2(const __grid_constant__ PassParams<T> pp) {
    constexpr int E = FastPlan<N>::E;
    constexpr int TPL = N / E;
    constexpr int TL = FAST_THREADS / TPL;
    constexpr int NH = N / 2 + 1;
    constexpr int PH = (NH % 2 == 0) ? NH + 1 : NH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* H = (cpx<T>*)smem_raw;
    cpx<T>* b0 = H + 2 * TL * PH;
    cpx<T>* b1 = b0 + TL * SIdx<N, 1>::LP;
    const PassJob& job = pp.jobs[blockIdx.y];
    const cpx<T>* tw = (const cpx<T>*)pp.ax.tw;
    const int rows = pp.n0 * pp.n1;
    const int r0 = blockIdx.x * 2 * TL;
    const int nr = min(2 * TL, rows - r0);
    const int c = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const bool va = 2 * c < nr, vb = 2 * c + 1 < nr;
    cpx<T> x[E];
    if (pp.sign > 0) {
        for (int e = threadIdx.x; e < 2 * TL * NH; e += FAST_THREADS) {
            const int row = e % (2 * TL), k = e / (2 * TL);
            cpx<T> acc = mk((T)0, (T)0);
            if (row < nr)
                for (int b = 0; b < job.nin; ++b)
                    acc = acc + (T)job.isym[b].scale * ((const cpx<T>*)job.in[b])[(size_t)k * rows + r0 + row];
            H[row * PH + k] = acc;
        }
        for (int o = 0; o < job.nout; ++o) {
            const SymD sy = job.osym[o];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = t + TPL * m;
                const bool lo = k < NH;
                const int kk = lo ? k : N - k;
                cpx<T> a = sym_apply(sy, pp.tabs, 0, 0, kk, H[(2 * c) * PH + kk]);
                cpx<T> b = sym_apply(sy, pp.tabs, 0, 0, kk, H[(2 * c + 1) * PH + kk]);
                if (kk == 0 || kk == N / 2) {
                    a.y = 0;
                    b.y = 0;
                }
                if (!lo) {
                    a = cj(a);
                    b = cj(b);
                }
                x[m] = mk(a.x - b.y, a.y + b.x);
            }
            fast_fft<T, N, 1>(x, b0, b1, c, t, tw, +1);
            T* out = (T*)job.out[o];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int p = t + TPL * m;
                if (va) out[(size_t)(r0 + 2 * c) * N + p] = x[m].x;
                if (vb) out[(size_t)(r0 + 2 * c + 1) * N + p] = x[m].y;
            }
        }
    } else {
        for (int q = 0; q < job.nin; ++q) {
            const T* in = (const T*)job.in[q];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int p = t + TPL * m;
                const T a = va ? in[(size_t)(r0 + 2 * c) * N + p] : (T)0;
                const T b = vb ? in[(size_t)(r0 + 2 * c + 1) * N + p] : (T)0;
                x[m] = mk(a, b);
            }
            fast_fft<T, N, 1>(x, b0, b1, c, t, tw, -1);
            // stage the packed spectrum to pair Z_k with Z_{N-k}
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) b0[SIdx<N, 1>::at(c, t + TPL * m)] = x[m];
            __syncthreads();
            const SymD sy = job.isym[q];
            for (int k = t; k < NH; k += TPL) {
                const cpx<T> zk = b0[SIdx<N, 1>::at(c, k)];
                const cpx<T> zn = cj(b0[SIdx<N, 1>::at(c, k == 0 ? 0 : N - k)]);
                const cpx<T> sa = sym_apply(sy, pp.tabs, 0, 0, k, (T)0.5 * (zk + zn));
                const cpx<T> sb = sym_apply(sy, pp.tabs, 0, 0, k, rot((T)0.5 * (zk - zn), -1));
                cpx<T>* ha = &H[(2 * c) * PH + k];
                cpx<T>* hb = &H[(2 * c + 1) * PH + k];
                *ha = q == 0 ? sa : *ha + sa;
                *hb = q == 0 ? sb : *hb + sb;
            }
        }
        __syncthreads();
        cpx<T>* out = (cpx<T>*)job.out[0];
        for (int e = threadIdx.x; e < 2 * TL * NH; e += FAST_THREADS) {
            const int row = e % (2 * TL), k = e / (2 * TL);
            if (row < nr) out[(size_t)k * rows + r0 + row] = H[row * PH + k];
        }
    }
}

template <class T, int N> constexpr size_t fast_c2c_smem(int axis) {
    return (size_t)2 * (FAST_THREADS / (N / FastPlan<N>::E)) * (axis == 1 ? SIdx<N, 1>::LP : SIdx<N, 0>::LP) *
           sizeof(cpx<T>);
}
template <class T, int N> constexpr size_t fast_axis2_smem() {
    constexpr int TL = FAST_THREADS / (N / FastPlan<N>::E);
    constexpr int NH = N / 2 + 1;
    constexpr int PH = (NH % 2 == 0) ? NH + 1 : NH;
    return ((size_t)2 * TL * PH + (size_t)2 * TL * SIdx<N, 1>::LP) * sizeof(cpx<T>);
}

}  // namespace lddmm
