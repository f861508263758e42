// Pointwise kernels on real fields: the ad* / ad bilinear forms of the EPDiff
// equation and of the Jacobi sweeps, semi-Lagrangian transport (global-gather
// and shared-memory-staged map steps), warping, the exact transposes of the
// map step and of the warp (discrete gradient), Jacobian determinants and
// double-precision reductions.
//
// A time state holds 24 real fields, each N = n0*n1*n2 values:
//   [0..2]   v_c          [3 + 3c + j]  D_j v_c
//   [12..14] m_c = (L v)_c [15 + 3c + j] D_j m_c
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace lddmm {

constexpr int PW_THREADS = 256;

// Stored values are T or bfloat16 (the precision form's state storage); they
// are widened to the compute type on load.
template <class T> __device__ __forceinline__ T widen(T x) { return x; }
__device__ __forceinline__ float widen(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class S> struct StatePtr {
    const S* p;  // 24 fields, stride N
    size_t N;
    __device__ __forceinline__ auto v(int c, size_t x) const { return widen(p[c * N + x]); }
    __device__ __forceinline__ auto Dv(int c, int j, size_t x) const { return widen(p[(3 + 3 * c + j) * N + x]); }
    __device__ __forceinline__ auto m(int c, size_t x) const { return widen(p[(12 + c) * N + x]); }
    __device__ __forceinline__ auto Dm(int c, int j, size_t x) const { return widen(p[(15 + 3 * c + j) * N + x]); }
};

// ad*_v m = (Dv)^T m + (Dm) v + m div v  (EPDiff bracket, Sec. 2.2).
// With store != nullptr the 24 input fields are also written to the state
// store in bfloat16 (precision form).
template <class T>
__global__ void k_adstar(StatePtr<T> S, T* __restrict__ out, size_t N, __nv_bfloat16* __restrict__ store) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        T v[3], m[3], Dv[3][3], Dm[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = S.v(c, x);
            m[c] = S.m(c, x);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Dv[c][j] = S.Dv(c, j, x);
                Dm[c][j] = S.Dm(c, j, x);
            }
        }
        const T divv = Dv[0][0] + Dv[1][1] + Dv[2][2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T a = m[i] * divv;
#pragma unroll
            for (int j = 0; j < 3; ++j) a += Dv[j][i] * m[j] + Dm[i][j] * v[j];
            out[i * N + x] = a;
        }
        if (store) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                store[c * N + x] = __float2bfloat16_rn((float)v[c]);
                store[(12 + c) * N + x] = __float2bfloat16_rn((float)m[c]);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    store[(3 + 3 * c + j) * N + x] = __float2bfloat16_rn((float)Dv[c][j]);
                    store[(15 + 3 * c + j) * N + x] = __float2bfloat16_rn((float)Dm[c][j]);
                }
            }
        }
    }
}

// Tangent (forward Jacobi) stage, pointwise part:
//  p = ad*_eta m + ad*_v mu  (mu = L eta),   q = ad_v xi = (Dv) xi - (Dxi) v.
// E holds eta in the 24-field state layout (eta, D eta, mu, D mu);
// X holds xi (0..2) and D_j xi_c at 3 + 3c + j.
template <class T, class SS>
__global__ void k_tangent_pw(StatePtr<SS> S, StatePtr<T> E, const T* __restrict__ X, T* __restrict__ out, size_t N) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        T v[3], m[3], e[3], mu[3], xi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = S.v(c, x);
            m[c] = S.m(c, x);
            e[c] = E.v(c, x);
            mu[c] = E.m(c, x);
            xi[c] = X[c * N + x];
        }
        const T divv = S.Dv(0, 0, x) + S.Dv(1, 1, x) + S.Dv(2, 2, x);
        const T dive = E.Dv(0, 0, x) + E.Dv(1, 1, x) + E.Dv(2, 2, x);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T p = m[i] * dive + mu[i] * divv;
            T q = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                p += E.Dv(j, i, x) * m[j] + S.Dm(i, j, x) * e[j] + S.Dv(j, i, x) * mu[j] + E.Dm(i, j, x) * v[j];
                q += S.Dv(i, j, x) * xi[j] - X[(3 + 3 * i + j) * N + x] * v[j];
            }
            out[i * N + x] = p;
            out[(3 + i) * N + x] = q;
        }
    }
}

// Adjoint (transposed Jacobi) stage, pointwise part.  Inputs y = K ybar_eta
// and yx = ybar_xi (3 fields each).  Writes 9 groups of 4 fields
// [scalar s, f_0, f_1, f_2]; the forward transform of a group is
// F(s) + sum_j i kappa_j F(f_j):
//   group c     : R'^T part without L:  s = -sum_i D_c m_i y_i,  f_i = m_c y_i + delta_ic (m.y)
//   group 3 + c : R'^T part under -L:   s = sum_i D_i v_c y_i + (div v) y_c,  f_j = -v_j y_c
//   group 6 + c : ad_v^T yx:            s = sum_i D_c v_i yx_i,  f_j = v_j yx_c
template <class T, class SS>
__global__ void k_adjoint_pw(StatePtr<SS> S, const T* __restrict__ Y, T* __restrict__ out, size_t N) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        T v[3], m[3], y[3], yx[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = S.v(c, x);
            m[c] = S.m(c, x);
            y[c] = Y[c * N + x];
            yx[c] = Y[(3 + c) * N + x];
        }
        const T divv = S.Dv(0, 0, x) + S.Dv(1, 1, x) + S.Dv(2, 2, x);
        const T my = m[0] * y[0] + m[1] * y[1] + m[2] * y[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T s1 = 0, s2 = divv * y[c], s3 = 0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                s1 -= S.Dm(i, c, x) * y[i];
                s2 += S.Dv(c, i, x) * y[i];
                s3 += S.Dv(i, c, x) * yx[i];
            }
            T* g1 = out + (size_t)(4 * c) * N;
            T* g2 = out + (size_t)(4 * (3 + c)) * N;
            T* g3 = out + (size_t)(4 * (6 + c)) * N;
            g1[x] = s1;
            g2[x] = s2;
            g3[x] = s3;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                g1[(1 + j) * N + x] = m[c] * y[j] + (j == c ? my : (T)0);
                g2[(1 + j) * N + x] = -v[j] * y[c];
                g3[(1 + j) * N + x] = v[j] * yx[c];
            }
        }
    }
}

// ---------------------------------------------------------------- interpolation
struct GridI {
    int n0, n1, n2;
};

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

template <class T> __device__ __forceinline__ void cr_weights(T t, T* w) {
    const T t2 = t * t, t3 = t2 * t;
    w[0] = (T)0.5 * (-t3 + (T)2 * t2 - t);
    w[1] = (T)0.5 * ((T)3 * t3 - (T)5 * t2 + (T)2);
    w[2] = (T)0.5 * ((T)-3 * t3 + (T)4 * t2 + t);
    w[3] = (T)0.5 * (t3 - t2);
}

// Interpolate NC fields (stride N) at voxel (i0,i1,i2) + d (d in voxels).
template <class T, int NC>
__device__ __forceinline__ void interp_at(const T* __restrict__ f, size_t N, GridI g, int i0, int i1, int i2,
                                          const T d[3], int cubic, T* res) {
    int base[3];
    T w[3][4];
    const int ii[3] = {i0, i1, i2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T fl = floor(d[a]);
        const T t = d[a] - fl;
        base[a] = ii[a] + (int)fl;
        if (cubic) {
            cr_weights(t, w[a]);
        } else {
            w[a][0] = (T)1 - t;
            w[a][1] = t;
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) res[c] = 0;
    const int lo = cubic ? -1 : 0, cnt = cubic ? 4 : 2;
    for (int a0 = 0; a0 < cnt; ++a0) {
        const size_t o0 = (size_t)wrapi(base[0] + lo + a0, g.n0) * g.n1;
        for (int a1 = 0; a1 < cnt; ++a1) {
            const size_t o1 = (o0 + wrapi(base[1] + lo + a1, g.n1)) * g.n2;
            const T w01 = w[0][a0] * w[1][a1];
            for (int a2 = 0; a2 < cnt; ++a2) {
                const size_t o = o1 + wrapi(base[2] + lo + a2, g.n2);
                const T ww = w01 * w[2][a2];
#pragma unroll
                for (int c = 0; c < NC; ++c) res[c] += ww * __ldg(&f[c * N + o]);
            }
        }
    }
}

// One semi-Lagrangian step of the inverse-map displacement u (psi = x + u):
//   Xt = x - dt v1(x);  X = x - dt/2 (v1(x) + v0(Xt));  u1(x) = (X - x) + u0(X).
template <class T>
__global__ void k_sl_step(GridI g, const T* __restrict__ v0, const T* __restrict__ v1, const T* __restrict__ u0,
                          T* __restrict__ u1, T dt, T ih0, T ih1, T ih2, int cubic, size_t N) {
    const T ih[3] = {ih0, ih1, ih2};
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(x % g.n2);
        const int i1 = (int)((x / g.n2) % g.n1);
        const int i0 = (int)(x / ((size_t)g.n2 * g.n1));
        T w1[3], d[3], vt[3], ut[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w1[c] = v1[c * N + x];
            d[c] = -dt * w1[c] * ih[c];
        }
        interp_at<T, 3>(v0, N, g, i0, i1, i2, d, cubic, vt);
        T disp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            disp[c] = (T)-0.5 * dt * (w1[c] + vt[c]);
            d[c] = disp[c] * ih[c];
        }
        interp_at<T, 3>(u0, N, g, i0, i1, i2, d, cubic, ut);
#pragma unroll
        for (int c = 0; c < 3; ++c) u1[c * N + x] = disp[c] + ut[c];
    }
}

// ---------------------------------------------------------------- staged map step (FP32)
// The map step of k_sl_step with its two gathers served from shared memory.
// A block owns an SLT0 x SLT1 x SLT2 tile of output points.  It stages the
// sampled field (first v0, then u0) over the tile plus a halo of LO / HI
// voxels as one float4 (x, y, z, 0) per grid point, so that a tap is one
// 16-byte shared load instead of three scalar global loads.  A point whose
// stencil leaves the staged box (more than SL_DMAX voxels of displacement in
// the step) takes the global gather of interp_at instead, so any velocity is
// handled; the taps and their summation order are those of interp_at.
constexpr int SLT0 = 4, SLT1 = 8, SLT2 = 32;  // threads: SLT1 * SLT2 = 256, SLT0 points each
constexpr int SL_DMAX = 1;                    // staged displacement per step, voxels
template <bool CUBIC> struct SLBox {
    static constexpr int TLO = CUBIC ? -1 : 0, CNT = CUBIC ? 4 : 2;  // tap offsets TLO .. TLO + CNT - 1
    static constexpr int LO = SL_DMAX - TLO;                         // halo below the tile
    static constexpr int HI = SL_DMAX + TLO + CNT - 1;               // halo above the tile
    static constexpr int B0 = SLT0 + LO + HI, B1 = SLT1 + LO + HI, B2 = SLT2 + LO + HI;
    static constexpr int SIZE = B0 * B1 * B2;
    static constexpr size_t SMEM = (size_t)SIZE * sizeof(float4);
};

// stage the 3 planes of f over the box whose corner is (c0, c1, c2), periodic
template <bool CUBIC>
__device__ __forceinline__ void sl_stage(float4* S, const float* __restrict__ f, size_t N, GridI g, int c0, int c1,
                                         int c2) {
    using B = SLBox<CUBIC>;
    // box coordinates lie in [-LO, n + B - LO): within one period of the grid
    // when n >= B, so one compare and add wraps them; smaller grids take the
    // general modulo
    const bool near = g.n0 >= B::B0 && g.n1 >= B::B1 && g.n2 >= B::B2;
    auto wrap = [near](int x, int n) { return near ? (x < 0 ? x + n : (x >= n ? x - n : x)) : wrapi(x, n); };
    for (int e = threadIdx.x; e < B::SIZE; e += SLT1 * SLT2) {
        const int b2 = e % B::B2, b1 = (e / B::B2) % B::B1, b0 = e / (B::B2 * B::B1);
        const size_t o = ((size_t)wrap(c0 + b0, g.n0) * g.n1 + wrap(c1 + b1, g.n1)) * g.n2 + wrap(c2 + b2, g.n2);
        S[e] = make_float4(__ldg(&f[o]), __ldg(&f[N + o]), __ldg(&f[2 * N + o]), 0.f);
    }
}

// the 3 components of the interpolant at (i0,i1,i2) + d: from the staged box
// when the whole stencil lies in it, else from global memory
template <bool CUBIC>
__device__ __forceinline__ void sl_interp(const float4* S, const float* __restrict__ f, size_t N, GridI g, int i0,
                                          int i1, int i2, int c0, int c1, int c2, const float d[3], float* res) {
    using B = SLBox<CUBIC>;
    int base[3];
    float w[3][4];
    const int ii[3] = {i0, i1, i2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(d[a]);
        const float t = d[a] - fl;
        base[a] = ii[a] + (int)fl;
        if constexpr (CUBIC) {
            cr_weights(t, w[a]);
        } else {
            w[a][0] = 1.f - t;
            w[a][1] = t;
        }
    }
    const int l0 = base[0] + B::TLO - c0, l1 = base[1] + B::TLO - c1, l2 = base[2] + B::TLO - c2;
    const bool inside = l0 >= 0 && l1 >= 0 && l2 >= 0 && l0 + B::CNT <= B::B0 && l1 + B::CNT <= B::B1 &&
                        l2 + B::CNT <= B::B2;
    if (!inside) {
        interp_at<float, 3>(f, N, g, i0, i1, i2, d, CUBIC ? 1 : 0, res);
        return;
    }
    res[0] = res[1] = res[2] = 0.f;
#pragma unroll
    for (int a0 = 0; a0 < B::CNT; ++a0) {
#pragma unroll
        for (int a1 = 0; a1 < B::CNT; ++a1) {
            const float w01 = w[0][a0] * w[1][a1];
            const float4* row = S + ((l0 + a0) * B::B1 + (l1 + a1)) * B::B2 + l2;
#pragma unroll
            for (int a2 = 0; a2 < B::CNT; ++a2) {
                const float ww = w01 * w[2][a2];
                const float4 v = row[a2];
                res[0] += ww * v.x;
                res[1] += ww * v.y;
                res[2] += ww * v.z;
            }
        }
    }
}

// k_sl_step for FP32 with staged gathers: grid (ceil(n2/SLT2), ceil(n1/SLT1),
// ceil(n0/SLT0)), SLT1 * SLT2 threads, SLBox<CUBIC>::SMEM dynamic shared bytes
template <bool CUBIC>
__global__ void __launch_bounds__(SLT1* SLT2) k_sl_step_staged(GridI g, const float* __restrict__ v0,
                                                               const float* __restrict__ v1,
                                                               const float* __restrict__ u0, float* __restrict__ u1,
                                                               float dt, float ih0, float ih1, float ih2, size_t N) {
    using B = SLBox<CUBIC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* S = (float4*)smem_raw;
    const float ih[3] = {ih0, ih1, ih2};
    const int o0 = blockIdx.z * SLT0, o1 = blockIdx.y * SLT1, o2 = blockIdx.x * SLT2;
    const int i1 = o1 + threadIdx.x / SLT2, i2 = o2 + threadIdx.x % SLT2;
    const int c0 = o0 - B::LO, c1 = o1 - B::LO, c2 = o2 - B::LO;  // box corner
    const bool col = i1 < g.n1 && i2 < g.n2;
    float disp[SLT0][3];
    sl_stage<CUBIC>(S, v0, N, g, c0, c1, c2);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < SLT0; ++p) {
        const int i0 = o0 + p;
        if (!col || i0 >= g.n0) continue;
        const size_t x = ((size_t)i0 * g.n1 + i1) * g.n2 + i2;
        float w1[3], d[3], vt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w1[c] = v1[c * N + x];
            d[c] = -dt * w1[c] * ih[c];
        }
        sl_interp<CUBIC>(S, v0, N, g, i0, i1, i2, c0, c1, c2, d, vt);
#pragma unroll
        for (int c = 0; c < 3; ++c) disp[p][c] = -0.5f * dt * (w1[c] + vt[c]);
    }
    __syncthreads();
    sl_stage<CUBIC>(S, u0, N, g, c0, c1, c2);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < SLT0; ++p) {
        const int i0 = o0 + p;
        if (!col || i0 >= g.n0) continue;
        const size_t x = ((size_t)i0 * g.n1 + i1) * g.n2 + i2;
        float d[3], ut[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = disp[p][c] * ih[c];
        sl_interp<CUBIC>(S, u0, N, g, i0, i1, i2, c0, c1, c2, d, ut);
#pragma unroll
        for (int c = 0; c < 3; ++c) u1[c * N + x] = disp[p][c] + ut[c];
    }
}

// m(x) = I(x + u(x))
template <class T>
__global__ void k_warp(GridI g, const T* __restrict__ img, const T* __restrict__ u, T* __restrict__ out, T ih0, T ih1,
                       T ih2, int cubic, size_t N) {
    const T ih[3] = {ih0, ih1, ih2};
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(x % g.n2);
        const int i1 = (int)((x / g.n2) % g.n1);
        const int i0 = (int)(x / ((size_t)g.n2 * g.n1));
        T d[3], r[1];
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = u[c * N + x] * ih[c];
        interp_at<T, 1>(img, N, g, i0, i1, i2, d, cubic, r);
        out[x] = r[0];
    }
}

// ---------------------------------------------------------------- exact adjoint of the transport
// Interpolation weights w and their coordinate derivatives dw for one point.
template <class T> __device__ __forceinline__ void cr_dweights(T t, T* dw) {
    const T t2 = t * t;
    dw[0] = (T)0.5 * ((T)-3 * t2 + (T)4 * t - (T)1);
    dw[1] = (T)0.5 * ((T)9 * t2 - (T)10 * t);
    dw[2] = (T)0.5 * ((T)-9 * t2 + (T)8 * t + (T)1);
    dw[3] = (T)0.5 * ((T)3 * t2 - (T)2 * t);
}
// Taps of one point for the Catmull-Rom (CUBIC) or trilinear interpolant,
// with the tap count known at compile time (the weight arrays stay in
// registers).
template <class T, bool CUBIC> struct Taps {
    static constexpr int CNT = CUBIC ? 4 : 2;
    static constexpr int LO = CUBIC ? -1 : 0;
    int base[3];
    T w[3][CNT], dw[3][CNT];
    __device__ __forceinline__ Taps(int i0, int i1, int i2, const T d[3]) {
        const int ii[3] = {i0, i1, i2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T fl = floor(d[a]);
            const T t = d[a] - fl;
            base[a] = ii[a] + (int)fl;
            if constexpr (CUBIC) {
                cr_weights(t, w[a]);
                cr_dweights(t, dw[a]);
            } else {
                w[a][0] = (T)1 - t;
                w[a][1] = t;
                dw[a][0] = (T)-1;
                dw[a][1] = (T)1;
            }
        }
    }
};

// d/dp_b of the interpolant of NC fields at the point: G[b][c]
template <class T, bool CUBIC, int NC>
__device__ __forceinline__ void interp_grad_at(const T* __restrict__ f, size_t N, GridI g, const Taps<T, CUBIC>& tp,
                                               T (&G)[3][NC]) {
    constexpr int CNT = Taps<T, CUBIC>::CNT, LO = Taps<T, CUBIC>::LO;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NC; ++c) G[b][c] = 0;
#pragma unroll
    for (int a0 = 0; a0 < CNT; ++a0) {
        const size_t o0 = (size_t)wrapi(tp.base[0] + LO + a0, g.n0) * g.n1;
#pragma unroll
        for (int a1 = 0; a1 < CNT; ++a1) {
            const size_t o1 = (o0 + wrapi(tp.base[1] + LO + a1, g.n1)) * g.n2;
#pragma unroll
            for (int a2 = 0; a2 < CNT; ++a2) {
                const size_t o = o1 + wrapi(tp.base[2] + LO + a2, g.n2);
                const T g0 = tp.dw[0][a0] * tp.w[1][a1] * tp.w[2][a2];
                const T g1 = tp.w[0][a0] * tp.dw[1][a1] * tp.w[2][a2];
                const T g2 = tp.w[0][a0] * tp.w[1][a1] * tp.dw[2][a2];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T val = __ldg(&f[c * N + o]);
                    G[0][c] += g0 * val;
                    G[1][c] += g1 * val;
                    G[2][c] += g2 * val;
                }
            }
        }
    }
}

// Transpose of the interpolation at the point: fb[taps] += w * vals (atomic)
template <class T, bool CUBIC, int NC>
__device__ __forceinline__ void interp_scatter_at(T* fb, size_t N, GridI g, const Taps<T, CUBIC>& tp,
                                                  const T (&vals)[NC]) {
    constexpr int CNT = Taps<T, CUBIC>::CNT, LO = Taps<T, CUBIC>::LO;
#pragma unroll
    for (int a0 = 0; a0 < CNT; ++a0) {
        const size_t o0 = (size_t)wrapi(tp.base[0] + LO + a0, g.n0) * g.n1;
#pragma unroll
        for (int a1 = 0; a1 < CNT; ++a1) {
            const size_t o1 = (o0 + wrapi(tp.base[1] + LO + a1, g.n1)) * g.n2;
            const T w01 = tp.w[0][a0] * tp.w[1][a1];
#pragma unroll
            for (int a2 = 0; a2 < CNT; ++a2) {
                const size_t o = o1 + wrapi(tp.base[2] + LO + a2, g.n2);
                const T ww = w01 * tp.w[2][a2];
#pragma unroll
                for (int c = 0; c < NC; ++c) atomicAdd(&fb[c * N + o], ww * vals[c]);
            }
        }
    }
}

// Cotangent of the final warp m1 = I0(x + u/h) with respect to u, for
// E_data = ||m1 - I1||^2:  ub(x) = 2 (m1 - I1)(x) dI0/dp(x + u/h) / h.
template <class T, bool CUBIC>
__global__ void k_warp_adj(GridI g, const T* __restrict__ img, const T* __restrict__ u, const T* __restrict__ m1,
                           const T* __restrict__ I1, T* __restrict__ ub, T ih0, T ih1, T ih2, size_t N) {
    const T ih[3] = {ih0, ih1, ih2};
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(x % g.n2);
        const int i1 = (int)((x / g.n2) % g.n1);
        const int i0 = (int)(x / ((size_t)g.n2 * g.n1));
        T d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = u[c * N + x] * ih[c];
        const Taps<T, CUBIC> tp(i0, i1, i2, d);
        T G[3][1];
        interp_grad_at<T, CUBIC, 1>(img, N, g, tp, G);
        const T r2 = (T)2 * (m1[x] - I1[x]);
#pragma unroll
        for (int b = 0; b < 3; ++b) ub[b * N + x] = r2 * G[b][0] * ih[b];
    }
}

// Transpose of one map step (k_sl_step) u_{k+1} = disp + u_k(X),
// X = x + disp/h, disp = -dt/2 (v1 + v0(p1)), p1 = x - dt v1/h:
// from ub1 = dE/du_{k+1}, scatter dE/du_k into ub0 and the v0(p1) part of
// dE/dv_k into vb0 (both atomic), and add the v1 part of dE/dv_{k+1} to vb1.
template <class T, bool CUBIC>
__global__ void k_sl_adj(GridI g, const T* __restrict__ v0, const T* __restrict__ v1, const T* __restrict__ u0,
                         const T* __restrict__ ub1, T* ub0, T* vb0, T* __restrict__ vb1, T dt, T ih0, T ih1, T ih2,
                         size_t N) {
    const T ih[3] = {ih0, ih1, ih2};
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(x % g.n2);
        const int i1 = (int)((x / g.n2) % g.n1);
        const int i0 = (int)(x / ((size_t)g.n2 * g.n1));
        T w1[3], d1[3], vt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w1[c] = v1[c * N + x];
            d1[c] = -dt * w1[c] * ih[c];
        }
        interp_at<T, 3>(v0, N, g, i0, i1, i2, d1, CUBIC ? 1 : 0, vt);
        T dX[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) dX[c] = (T)-0.5 * dt * (w1[c] + vt[c]) * ih[c];
        const Taps<T, CUBIC> tX(i0, i1, i2, dX);
        T Gu[3][3];
        interp_grad_at<T, CUBIC, 3>(u0, N, g, tX, Gu);
        T ub[3], dispb[3], vtb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) ub[c] = ub1[c * N + x];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            dispb[b] = ub[b] + ih[b] * (Gu[b][0] * ub[0] + Gu[b][1] * ub[1] + Gu[b][2] * ub[2]);
            vtb[b] = (T)-0.5 * dt * dispb[b];
        }
        interp_scatter_at<T, CUBIC, 3>(ub0, N, g, tX, ub);
        const Taps<T, CUBIC> t1(i0, i1, i2, d1);
        interp_scatter_at<T, CUBIC, 3>(vb0, N, g, t1, vtb);
        T Gv[3][3];
        interp_grad_at<T, CUBIC, 3>(v0, N, g, t1, Gv);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T p1b = Gv[b][0] * vtb[0] + Gv[b][1] * vtb[1] + Gv[b][2] * vtb[2];
            vb1[b * N + x] += (T)-0.5 * dt * dispb[b] - dt * ih[b] * p1b;
        }
    }
}

// ---------------------------------------------------------------- reductions
// Deterministic two-phase double reductions: block partials, then one block.
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 592;  // 4 x 148..152 SMs; partial buffer size

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// op: 0 sum, 1 max, 2 min
__device__ __forceinline__ double block_reduce(double v, int op) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = op == 0 ? warp_sum(v) : (op == 1 ? warp_max(v) : warp_min(v));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    const double id = op == 0 ? 0.0 : (op == 1 ? -1.0e300 : 1.0e300);
    v = threadIdx.x < nw ? sh[threadIdx.x] : id;
    if (wid == 0) v = op == 0 ? warp_sum(v) : (op == 1 ? warp_max(v) : warp_min(v));
    __syncthreads();
    return v;
}

// partial[b] = sum over this block's share of a[x]*b[x] (b == nullptr: a[x]^2)
template <class T>
__global__ void k_dot_partial(const T* __restrict__ a, const T* __restrict__ b, size_t n, double* __restrict__ partial) {
    double acc = 0.0;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        const double av = (double)a[x];
        acc += av * (b ? (double)b[x] : av);
    }
    acc = block_reduce(acc, 0);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// partial[3*b + {0,1,2}] = {max|a|, max a, min a}
template <class T>
__global__ void k_absmax_partial(const T* __restrict__ a, size_t n, double* __restrict__ partial) {
    double am = 0.0, mx = -1.0e300, mn = 1.0e300;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)a[x];
        am = fmax(am, fabs(v));
        mx = fmax(mx, v);
        mn = fmin(mn, v);
        if (v != v) am = 1.0e308;  // NaN poisons max|a|
    }
    am = block_reduce(am, 1);
    mx = block_reduce(mx, 1);
    mn = block_reduce(mn, 2);
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x] = am;
        partial[3 * blockIdx.x + 1] = mx;
        partial[3 * blockIdx.x + 2] = mn;
    }
}

// Non-finite scan of up to SCAN_MAX arrays: *flag = 1 when any entry is a
// NaN or an infinity (the flag is never cleared; the caller's status is
// sticky).  The result does not depend on the launch shape.
constexpr int SCAN_MAX = 4;
template <class T> struct ScanArgs {
    const T* p[SCAN_MAX];
    size_t n[SCAN_MAX];
    int cnt;
};
template <class T>
__global__ void k_nonfinite_scan(const __grid_constant__ ScanArgs<T> a, double* __restrict__ flag) {
    bool bad = false;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int i = 0; i < a.cnt; ++i)
        for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < a.n[i]; x += stride)
            bad |= !isfinite(a.p[i][x]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1.0;
}

// out[slot] = scale * reduce(partial[0..nb*stride) with the given stride/offset)
static __global__ void k_finish(const double* __restrict__ partial, int nb, int stride, int off, int op, double scale,
                         double* __restrict__ out) {
    const double id = op == 0 ? 0.0 : (op == 1 ? -1.0e300 : 1.0e300);
    double v = id;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double p = partial[i * stride + off];
        v = op == 0 ? v + p : (op == 1 ? fmax(v, p) : fmin(v, p));
    }
    v = block_reduce(v, op);
    if (threadIdx.x == 0) *out = scale * v;
}

// ---------------------------------------------------------------- small pointwise ops
// y = a*x + b*y  over n values
template <class T>
__global__ void k_axpby(T a, const T* __restrict__ x, T b, T* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
// z = a*x + b*y
template <class T>
__global__ void k_lincomb2(T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* __restrict__ z, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        z[i] = a * x[i] + b * y[i];
}

// Final-time sources.  mode 0 (gradient):  out_c = -2 (m1 - I1) grad_c m1
//                      mode 1 (Gauss-Newton): out_c = 2 (grad m1 . xi) grad_c m1
template <class T>
__global__ void k_final_source(const T* __restrict__ m1, const T* __restrict__ I1, const T* __restrict__ gm,
                               const T* __restrict__ xi, T* __restrict__ out, int mode, size_t N) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const T g0 = gm[x], g1 = gm[N + x], g2 = gm[2 * N + x];
        T f;
        if (mode == 0) f = (T)-2 * (m1[x] - I1[x]);
        else f = (T)2 * (g0 * xi[x] + g1 * xi[N + x] + g2 * xi[2 * N + x]);
        out[x] = f * g0;
        out[N + x] = f * g1;
        out[2 * N + x] = f * g2;
    }
}

// Source of the shooting vector-Jacobian product: out_c = -G grad_c m1
template <class T>
__global__ void k_vjp_source(const T* __restrict__ G, const T* __restrict__ gm, T* __restrict__ out, size_t N) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const T g = -G[x];
        out[x] = g * gm[x];
        out[N + x] = g * gm[N + x];
        out[2 * N + x] = g * gm[2 * N + x];
    }
}

// r = m1 - I1
template <class T>
__global__ void k_sub(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ r, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        r[i] = a[i] - b[i];
}

// det(I + Du), Du[c][j] = D_j u_c at field 3c + j
template <class T>
__global__ void k_jacdet(const T* __restrict__ Du, T* __restrict__ J, size_t N) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        T a[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 3; ++j) a[c][j] = Du[(3 * c + j) * N + x] + (c == j ? (T)1 : (T)0);
        J[x] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
               a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    }
}

// Spectral-space combination on [k2][k0][k1] arrays: out = sum_b sym_b . in_b
template <class T> struct SpecComb {
    const cpx<T>* in[MAXI];
    SymT<T> sym[MAXI];
    int nin;
};
// A block walks (k2, k0) rows of n1 entries; its threads take the k1 of a
// row, so that the frequency indices cost one division per row.
template <class T>
__global__ void k_spec_comb(SpecComb<T> sc, SpecTabs<T> tb, int n0, int n1, int n2h, cpx<T>* __restrict__ out) {
    const int rows = n0 * n2h;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int k2 = r / n0, k0 = r - k2 * n0;
        const size_t base = (size_t)r * n1;
        for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) {
            const size_t x = base + k1;
            cpx<T> acc = mk((T)0, (T)0);
            for (int b = 0; b < sc.nin; ++b) acc = acc + sym_apply(sc.sym[b], tb, k0, k1, k2, sc.in[b][x]);
            out[x] = acc;
        }
    }
}
// launch shape of k_spec_comb: threads per block (whole warps covering a row, at most 256), blocks
inline int spec_comb_threads(int n1) { return n1 >= 256 ? 256 : ((n1 + 31) / 32) * 32; }
inline int spec_comb_blocks(int n0, int n2h) { return n0 * n2h < 152 * 16 ? n0 * n2h : 152 * 16; }

}  // namespace lddmm
