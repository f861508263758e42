// Fused Jacobi stages (FP32 form, band-limited transforms).
//
// One stage of the tangent sweep (Sec. 3, incremental EPDiff and Jacobi
// field) is: an inverse transform of (eta, xi) into 36 real fields, the
// pointwise products p = ad*_eta m + ad*_v mu, q = ad_v xi with the stored
// state, and a forward transform of (p, q).  One stage of the adjoint sweep
// (its exact transpose) is: an inverse transform into the 6 fields
// (K ybar_eta, P ybar_xi), the 36 pointwise group fields of the transposed
// products, and their forward transforms.  The axis-0 and axis-1 passes stay
// as they are; these kernels replace, for a tile of grid rows, the axis-2
// pass of the inverse transform, the pointwise kernel and the axis-2 pass of
// the forward transform, so that the real fields of a stage never leave the
// SM: each grid row is held by one line group of threads from its first
// inverse line transform to its last forward one.
//
// Geometry (register-blocked plans with E = 8 elements per thread):
//   a block of FAST_THREADS threads is TL line groups of TPL = N / 8 threads;
//   a tile is TL consecutive grid rows, one per line group; thread t of a
//   group owns the points t + TPL*m (m < 8) of its row for the whole tile.
//   A complex line transform packs two real fields of the same row.
//   Inputs and outputs are band planes k2 < NB2 in the [k2][row] layout of
//   the axis-2 pass; the next line's inputs are copied (cp.async) into the
//   other half of a double buffer while the current line is transformed.
//
// Tangent (KIND 0): inputs in[27], axis-1 outputs of the inverse transform,
//   for c = 0..2:  in[6c + 0] eta_c (gives eta_c and D2 eta_c),
//                  in[6c + 1], in[6c + 2] D0 eta_c, D1 eta_c,
//                  in[6c + 3] mu_c = (L eta)_c (gives mu_c and D2 mu_c),
//                  in[6c + 4], in[6c + 5] D0 mu_c, D1 mu_c,
//                  in[18 + 3c] xi_c (gives xi_c and D2 xi_c),
//                  in[19 + 3c], in[20 + 3c] D0 xi_c, D1 xi_c;
//   18 inverse line transforms per row accumulate p and q in registers;
//   outputs out[0..5] = F2(p_0..2), F2(q_0..2), the plain axis-2 transforms.
// Adjoint (KIND 1): inputs in[0..2] = K ybar_eta (y), in[3..5] = P ybar_xi
//   (yx); y and yx are kept in registers; the
//   9 groups (s, f_0, f_1, f_2) of the transposed products give 27 outputs,
//   for c = 0..2 and group g = 0 (R'^T without L), 1 (R'^T under -L),
//   2 (ad_v^T):  out[9c + 3g] = F2(s) + i kappa_2 F2(f_2),
//                out[9c + 3g + 1] = F2(f_0), out[9c + 3g + 2] = F2(f_1);
//   optional real cotangents eta_src (3 fields) are added to s of group 0.
//   Its inverse lines and its (s, f_2) forward lines pack two rows of one
//   field, as the separate axis-2 pass does (fields of one row can differ
//   widely in size, and a transform that packed s with f_2 would leave the
//   rounding of the larger in the smaller, which i kappa_2 then amplifies):
//   those fields are handed between the row's owner and the row pair's line
//   group through shared memory.  Its (f_0, f_1) forward lines, fields of
//   one group alike in size, pack the two fields of the owner's row.
#pragma once
#include "fft_fast.cuh"
#include "pw_kernels.cuh"

namespace lddmm {

constexpr int FUSED_NIN = 27, FUSED_NOUT = 27;
constexpr int FUSED_BLOCKS = 2;  // resident blocks per SM

struct FusedArgs {
    const cpx<float>* in[FUSED_NIN];
    cpx<float>* out[FUSED_NOUT];
    const void* states;     // 24 state fields (float or bfloat16), stride npts
    const float* eta_src;   // adjoint: 3 real fields added to s of group 0, or null
    const float* dk2;       // kappa_2 with the Nyquist entry zeroed (n2/2 + 1)
    const cpx<float>* tw;   // axis-2 twiddles
    int rows, nb2, ntiles;
    unsigned npts;          // points per field
};

template <int N> struct FusedGeom {
    static_assert(FastPlan<N>::E == 8, "fused stages use the E = 8 plans");
    static constexpr int E = 8;
    static constexpr int TPL = N / E;
    static constexpr int TL = FAST_THREADS / TPL;  // rows per tile
    static constexpr int NH = N / 2 + 1;
    static constexpr int SP = TL + 2;              // staged plane pitch (complex; 16-byte rows)
    static constexpr int XT = TL * SIdx<float, N, 1>::LP;  // one exchange tile
    // band planes of the dealiased grid: |k2| <= (N - 1) / 3 (the 2/3 rule of
    // the projector P); the stages run only on dealiased grids
    static constexpr int NB2 = (N - 1) / 3 + 1;
    static constexpr int PH = (NB2 % 2 == 0) ? NB2 + 1 : NB2;  // H pitch (odd: conflict-free columns)
    static constexpr int HS = 2 * TL * PH;         // two unpacked outputs (band planes)
    static constexpr int CPK = TL * 8 / 16;        // 16-byte chunks per staged plane
    // adjoint hand-off of two real fields: row pitch RP and field stride FS
    // (floats), both 16 banks apart modulo 32, so that neither the two rows
    // nor the two fields a warp touches share a bank
    static constexpr int RP = N + 16;
    static constexpr int FS = TL * RP + 16;
    static constexpr int TWD = N + (NH + 1) / 2;   // twiddles, then kappa_2 (complex slots)
    // Shared memory: two stage buffers, each the band planes k2 < NB2 of two
    // inputs and at least HS (the forward lines' unpacked outputs H live in
    // the buffer that no copy targets then), one exchange tile (shared by
    // every exchange of a line transform), the tables, and for the adjoint
    // the hand-off rows.  What it leaves of the SM's 256 KB serves as L1 for
    // the prefetched states.
    // exchanges addressed by XOR (XorEx): every tile starts on a line-size
    // (8 N byte) boundary of the shared window
    static constexpr bool XA = XorEx<float, N>::ok;
    static constexpr int XAL = XA ? N * (int)sizeof(cpx<float>) : 16;
    static constexpr int STG0 = 2 * NB2 * SP > HS ? 2 * NB2 * SP : HS;
    static constexpr int STG = XA ? (STG0 + N - 1) / N * N : STG0;
    static constexpr size_t smem(int kind) {
        return (size_t)(XAL - 16) + (size_t)(2 * STG + XT + TWD) * sizeof(cpx<float>) +
               (kind == 1 ? (size_t)2 * FS * sizeof(float) : 0);
    }
    static_assert(TL % 2 == 0, "the adjoint pairs the rows of a tile");
    static_assert(!XA || (STG % N == 0 && XT % N == 0), "exchange tiles on line-size boundaries");
};

__device__ __forceinline__ float ldst(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldst(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// Stored-state field f of this thread's point m (state layout of pw_kernels.cuh)
template <class SS> struct PtState {
    const SS* p;  // this thread's first point of field 0
    unsigned n;   // field stride
    __device__ __forceinline__ float operator()(int f, int m, int tpl) const { return ldst(p + f * n + tpl * m); }
};
// field indices
__device__ __forceinline__ constexpr int fV(int c) { return c; }
__device__ __forceinline__ constexpr int fDv(int c, int j) { return 3 + 3 * c + j; }  // D_j v_c
__device__ __forceinline__ constexpr int fM(int c) { return 12 + c; }
__device__ __forceinline__ constexpr int fDm(int c, int j) { return 15 + 3 * c + j; }  // D_j m_c

// The q-th state field that line (c, type) reads (-1 past the last), the
// same for the tangent's inverse lines and the adjoint's forward lines (see
// tan_contrib and adj_fields); at most 6.
__device__ __forceinline__ int line_field(int c, int ty, int q) {
    switch (ty) {
        case 0:  // D_c m_0..2, m_c (and m_0, m_1 for c = 2)
            if (q < 3) return fDm(q, c);
            if (q == 3) return fM(c);
            return c == 2 && q < 6 ? fM(q - 4) : -1;
        case 1:  // m_c (and every m_k for c < 2)
            if (c == 2) return q == 0 ? fM(2) : -1;
            return q < 3 ? fM(q) : -1;
        case 2:  // D_0..2 v_c, the other two diagonal entries of D v, v_2
            if (q < 3) return fDv(c, q);
            if (q < 5) {
                const int i = q - 3 + (q - 3 >= c ? 1 : 0);
                return fDv(i, i);
            }
            return q == 5 ? fV(2) : -1;
        case 4:  // D_c v_0..2, v_2
            if (q < 3) return fDv(q, c);
            return q == 3 ? fV(2) : -1;
        default:  // v_0, v_1
            return q < 2 ? fV(q) : -1;
    }
}

// Bring the state rows of a tile that line (c, type) reads into L1 (one
// prefetch per 128-byte line), ahead of the loads of its products, so that
// those loads do not wait on L2; with L2 = true, into L2 only (a line
// further ahead, so that the L1 prefetch does not wait on DRAM).
template <class SS, int N, int TL, bool L2 = false>
__device__ __forceinline__ void prefetch_line_fields(const SS* tile_states, unsigned npts, int c, int ty) {
    // the tile's rows of one field are contiguous: PER cache lines
    constexpr int PER = (int)(TL * N * sizeof(SS) / 128);
    static_assert(PER * 128 == TL * N * sizeof(SS), "whole cache lines per tile");
    for (int i = threadIdx.x; i < 6 * PER; i += FAST_THREADS) {
        const int f = line_field(c, ty, i / PER);
        if (f < 0) break;
        const char* p = (const char*)(tile_states + (size_t)f * npts) + (size_t)(i % PER) * 128;
        if constexpr (L2) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        else asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    }
}

// Tangent: contributions of inverse line L (c = L / 6, type L % 6) to
// acc = (p_0, p_1, p_2, q_0, q_1, q_2):
//   p_i = m_i div eta + mu_i div v + sum_j (D_i eta_j m_j + D_j m_i eta_j + D_i v_j mu_j + D_j mu_i v_j)
//   q_i = sum_j (D_j v_i xi_j - D_j xi_i v_j)
template <int L, int E, int TPL, class SS>
__device__ __forceinline__ void tan_contrib(float (&acc)[6][E], const cpx<float> (&x)[E], const PtState<SS>& S) {
    constexpr int C = L / 6, TY = L % 6;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const float a = x[m].x, b = x[m].y;
        if constexpr (TY == 0) {  // (eta_C, D_2 eta_C)
            acc[0][m] += S(fDm(0, C), m, TPL) * a;
            acc[1][m] += S(fDm(1, C), m, TPL) * a;
            acc[2][m] += S(fDm(2, C), m, TPL) * a;
            const float mC = S(fM(C), m, TPL);
            acc[2][m] += b * mC;
            if constexpr (C == 2) {
                acc[0][m] += S(fM(0), m, TPL) * b;
                acc[1][m] += S(fM(1), m, TPL) * b;
                acc[2][m] += mC * b;
            }
        } else if constexpr (TY == 1) {  // (D_0 eta_C, D_1 eta_C)
            const float mC = S(fM(C), m, TPL);
            acc[0][m] += a * mC;
            acc[1][m] += b * mC;
            if constexpr (C < 2) {
                const float dd = C == 0 ? a : b;  // D_C eta_C, a term of div eta
#pragma unroll
                for (int k = 0; k < 3; ++k) acc[k][m] += (k == C ? mC : S(fM(k), m, TPL)) * dd;
            }
        } else if constexpr (TY == 2) {  // (mu_C, D_2 mu_C)
#pragma unroll
            for (int i = 0; i < 3; ++i) acc[i][m] += S(fDv(C, i), m, TPL) * a;
            const float divv = S(fDv(0, 0), m, TPL) + S(fDv(1, 1), m, TPL) + S(fDv(2, 2), m, TPL);
            acc[C][m] += a * divv;
            acc[C][m] += b * S(fV(2), m, TPL);
        } else if constexpr (TY == 3) {  // (D_0 mu_C, D_1 mu_C)
            acc[C][m] += a * S(fV(0), m, TPL);
            acc[C][m] += b * S(fV(1), m, TPL);
        } else if constexpr (TY == 4) {  // (xi_C, D_2 xi_C)
#pragma unroll
            for (int i = 0; i < 3; ++i) acc[3 + i][m] += S(fDv(i, C), m, TPL) * a;
            acc[3 + C][m] -= b * S(fV(2), m, TPL);
        } else {  // (D_0 xi_C, D_1 xi_C)
            acc[3 + C][m] -= a * S(fV(0), m, TPL);
            acc[3 + C][m] -= b * S(fV(1), m, TPL);
        }
    }
}

// Adjoint: the two real fields of forward line F (c = F / 6, type F % 6) from
// y = K ybar_eta = acc[0..2], yx = P ybar_xi = acc[3..5] and the state:
//   group 0:  s = -sum_i D_c m_i y_i,          f_j = m_c y_j + delta_jc (m . y)
//   group 1:  s = sum_i D_i v_c y_i + (div v) y_c,  f_j = -v_j y_c
//   group 2:  s = sum_i D_c v_i yx_i,          f_j = v_j yx_c
// even types pack (s, f_2), odd types (f_0, f_1).
template <int F, int E, int TPL, class SS>
__device__ __forceinline__ void adj_fields(cpx<float> (&x)[E], const float (&acc)[6][E], const PtState<SS>& S,
                                           const float* eta, unsigned npts) {
    constexpr int C = F / 6, TY = F % 6;
    const float(&y)[6][E] = acc;  // y_i = acc[i], yx_i = acc[3 + i]
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float a, b;
        if constexpr (TY == 0 || TY == 1) {
            const float mC = S(fM(C), m, TPL);
            float my = 0.f;
            if constexpr ((TY == 0 && C == 2) || (TY == 1 && C < 2))
                my = S(fM(0), m, TPL) * y[0][m] + S(fM(1), m, TPL) * y[1][m] + S(fM(2), m, TPL) * y[2][m];
            if constexpr (TY == 0) {
                a = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i) a -= S(fDm(i, C), m, TPL) * y[i][m];
                if (eta) a += __ldg(eta + C * npts + TPL * m);
                b = mC * y[2][m] + (C == 2 ? my : 0.f);
            } else {
                a = mC * y[0][m] + (C == 0 ? my : 0.f);
                b = mC * y[1][m] + (C == 1 ? my : 0.f);
            }
        } else if constexpr (TY == 2 || TY == 3) {
            if constexpr (TY == 2) {
                const float divv = S(fDv(0, 0), m, TPL) + S(fDv(1, 1), m, TPL) + S(fDv(2, 2), m, TPL);
                a = divv * y[C][m];
#pragma unroll
                for (int i = 0; i < 3; ++i) a += S(fDv(C, i), m, TPL) * y[i][m];
                b = -S(fV(2), m, TPL) * y[C][m];
            } else {
                a = -S(fV(0), m, TPL) * y[C][m];
                b = -S(fV(1), m, TPL) * y[C][m];
            }
        } else {
            if constexpr (TY == 4) {
                a = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i) a += S(fDv(i, C), m, TPL) * y[3 + i][m];
                b = S(fV(2), m, TPL) * y[3 + C][m];
            } else {
                a = S(fV(0), m, TPL) * y[3 + C][m];
                b = S(fV(1), m, TPL) * y[3 + C][m];
            }
        }
        x[m] = mk(a, b);
    }
}

// Element m of thread t of a line (k = t + TPL m) in a C2R line transform
// that packs two real rows (u, v) as u + i v: the half-spectrum index kk it
// reads (k, or N - k with conjugation above N / 2) and whether the entry is
// one of the real ones (k = 0, N / 2).  With E = 8 the element's range is
// known from m: m < 4 below N / 2, m = 4 at N / 2 + t, m > 4 above.
template <int N, int TPL> struct HermIdx {
    int kk;
    bool conj, real;
    __device__ __forceinline__ HermIdx(int t, int m) {
        static_assert(N == 8 * TPL, "E = 8 plans");
        if (m < 4) {
            kk = t + TPL * m;
            conj = false;
            real = m == 0 && t == 0;
        } else if (m == 4) {
            kk = N / 2 - t;
            conj = t != 0;
            real = t == 0;
        } else {
            kk = N - TPL * m - t;
            conj = true;
            real = false;
        }
    }
    // the line's entry u + i v, u and v the rows' half-spectrum values at kk
    __device__ __forceinline__ cpx<float> pack(cpx<float> u, cpx<float> v) const {
        if (real) {
            u.y = 0.f;
            v.y = 0.f;
        }
        if (conj) {
            u = cj(u);
            v = cj(v);
        }
        return mk(u.x - v.y, u.y + v.x);
    }
};

// inputs of inverse line l: (i0, i1); i1 = -1: the line packs (in[i0],
// D2 in[i0]) (tangent only)
template <int KIND> __device__ __forceinline__ void fused_line_inputs(int l, int& i0, int& i1) {
    if constexpr (KIND == 0) {
        const int c = l / 6, ty = l - 6 * c;
        if (ty < 4) {
            i0 = 6 * c + (ty < 2 ? 0 : 3) + (ty & 1);
            i1 = (ty & 1) ? i0 + 1 : -1;
        } else {
            i0 = 18 + 3 * c + (ty - 4);
            i1 = ty == 5 ? i0 + 1 : -1;
        }
    } else {
        // (y0, y1), (y2, yx0), (yx1, yx2)
        i0 = 2 * l;
        i1 = 2 * l + 1;
    }
}

template <class SS, int N, int KIND>
__global__ void __launch_bounds__(FAST_THREADS, FUSED_BLOCKS) k_fused_stage(const __grid_constant__ FusedArgs a) {
    using G = FusedGeom<N>;
    constexpr int E = G::E, TPL = G::TPL, TL = G::TL, NH = G::NH, SP = G::SP, PH = G::PH, RP = G::RP, FS = G::FS;
    constexpr int NLI = KIND == 0 ? 18 : 3;   // inverse lines per row (tangent) / rounds (adjoint)
    constexpr int NLO = KIND == 0 ? 3 : 18;   // forward lines per row / rounds
    constexpr int NBUF = 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int STG = G::STG;                         // one stage buffer (complex)
    constexpr bool XA = G::XA;
    cpx<float>* const stage0 = (cpx<float>*)align_smem<G::XAL>(smem_raw);  // buffers stage0 + sb * STG, sb < NBUF
    cpx<float>* const b0 = stage0 + NBUF * STG;
    cpx<float>* const tws = b0 + G::XT;                 // twiddles
    float* const dks = (float*)(tws + N);              // kappa_2 (Nyquist zeroed)
    float* const R = (float*)(tws + G::TWD);           // adjoint: two real fields of the tile's rows
    const int c = threadIdx.x / TPL, t = threadIdx.x % TPL;
    // adjoint: a line group transforms one field (q) on a pair of rows (2 rp, 2 rp + 1)
    const int q = c & 1, rp = c >> 1;
    constexpr int nb2 = G::NB2;
    const int rows = a.rows, ntiles = a.ntiles;

    auto issue = [&](int tile, int l, int buf) {
        if (tile < ntiles) {
            int i0, i1;
            fused_line_inputs<KIND>(l, i0, i1);
            const int nin = i1 >= 0 ? 2 : 1;  // staged inputs
            const int per = nb2 * G::CPK;
            cpx<float>* dst = stage0 + buf * STG;
            const size_t r0 = (size_t)tile * TL;
            for (int i = threadIdx.x; i < nin * per; i += FAST_THREADS) {
                const int qq = i >= per;
                const int rem = i - qq * per;
                const int k = rem / G::CPK, ch = rem % G::CPK;
                const cpx<float>* src = a.in[qq ? i1 : i0] + (size_t)k * rows + r0;
                cp_async16(dst + qq * nb2 * SP + k * SP + 2 * ch, src + 2 * ch);
            }
        }
        cp_async_commit();
    };

    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    static_assert(TwTable<N>::SIZE <= N, "per-stage twiddle tables fit N entries");
    fill_stage_twiddles<float, N>(tws, a.tw);
    for (int i = threadIdx.x; i < NH; i += FAST_THREADS) dks[i] = __ldg(a.dk2 + i);
    // the (tile, line) units of this block in order; the first NBUF - 1 go in
    // flight now, and each line sends the one NBUF - 1 ahead
    auto ahead = [&](int tl, int l, int d, int& tl2, int& l2) {
        tl2 = tl;
        l2 = l + d;
        while (l2 >= NLI) {
            l2 -= NLI;
            tl2 += gridDim.x;
        }
    };
    for (int d = 0; d < NBUF - 1; ++d) {
        int tl2, l2;
        ahead(tile, 0, d, tl2, l2);
        issue(tl2, l2, d);
    }
    int sb = 0;
    const SS* const states = (const SS*)a.states;
    cpx<float> x[E];
    for (; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * TL;
        const SS* const tile_states = states + (size_t)r0 * N;
        const PtState<SS> S{states + (size_t)(r0 + c) * N + t, a.npts};
        // tangent: p, q accumulators; adjoint: y, yx
        float acc[6][E];
#pragma unroll
        for (int f = 0; f < 6; ++f)
#pragma unroll
            for (int m = 0; m < E; ++m) acc[f][m] = 0.f;
        // ---------------- inverse lines
        for (int l = 0; l < NLI; ++l) {
            // this line's inputs are complete and visible, and every warp is
            // done with the other buffer (read by the previous line) before
            // the next line's copies go there
            cp_async_wait<NBUF - 2>();
            __syncthreads();
            {
                int tl2, l2;
                ahead(tile, l, NBUF - 1, tl2, l2);
                issue(tl2, l2, sb == 0 ? NBUF - 1 : sb - 1);
            }
            const cpx<float>* const stg = stage0 + sb * STG;
            if constexpr (KIND == 0) {
                prefetch_line_fields<SS, N, TL>(tile_states, a.npts, l / 6, l % 6);
                // two fields of this line group's row: (in[i0], D2 in[i0]) or (in[i0], in[i1])
                int i0, i1;
                fused_line_inputs<KIND>(l, i0, i1);
                const cpx<float>* SA = stg + c;
                if (i1 < 0) {
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        const HermIdx<N, TPL> h(t, m);
                        cpx<float> u = mk(0.f, 0.f), v = mk(0.f, 0.f);
                        if (h.kk < nb2) {
                            u = SA[h.kk * SP];
                            const float d = dks[h.kk];
                            v = mk(-d * u.y, d * u.x);
                        }
                        x[m] = h.pack(u, v);
                    }
                } else {
                    const cpx<float>* SB = SA + nb2 * SP;
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        const HermIdx<N, TPL> h(t, m);
                        cpx<float> u = mk(0.f, 0.f), v = mk(0.f, 0.f);
                        if (h.kk < nb2) {
                            u = SA[h.kk * SP];
                            v = SB[h.kk * SP];
                        }
                        x[m] = h.pack(u, v);
                    }
                }
            } else {
                if (l == NLI - 1) prefetch_line_fields<SS, N, TL>(tile_states, a.npts, 0, 0);
                // one field (input q of the line) on a pair of rows
                // the row pair's two entries are adjacent: one 16-byte load
                const float4* SA = (const float4*)(stg + q * nb2 * SP + 2 * rp);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const HermIdx<N, TPL> h(t, m);
                    float4 uv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (h.kk < nb2) uv = SA[h.kk * (SP / 2)];
                    x[m] = h.pack(mk(uv.x, uv.y), mk(uv.z, uv.w));
                }
            }
            fast_fft<float, N, 1, true, XA, true>(x, b0, b0, c, t, tws, +1);
            if constexpr (KIND == 0) {
                switch (l) {
#define LDDMM_TC(L) \
    case L: tan_contrib<L, E, TPL>(acc, x, S); break;
                    LDDMM_TC(0) LDDMM_TC(1) LDDMM_TC(2) LDDMM_TC(3) LDDMM_TC(4) LDDMM_TC(5)
                    LDDMM_TC(6) LDDMM_TC(7) LDDMM_TC(8) LDDMM_TC(9) LDDMM_TC(10) LDDMM_TC(11)
                    LDDMM_TC(12) LDDMM_TC(13) LDDMM_TC(14) LDDMM_TC(15) LDDMM_TC(16) LDDMM_TC(17)
#undef LDDMM_TC
                    default: break;
                }
            } else {
                // hand the row pair to the rows' owners: acc[2l], acc[2l + 1]
                float* const Rq = R + q * FS + 2 * rp * RP + t;
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    Rq[TPL * m] = x[m].x;
                    Rq[RP + TPL * m] = x[m].y;
                }
                __syncthreads();
                const float* const Ro = R + c * RP + t;
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const float f0 = Ro[TPL * m], f1 = Ro[FS + TPL * m];
                    if (l == 0) {
                        acc[0][m] = f0;
                        acc[1][m] = f1;
                    } else if (l == 1) {
                        acc[2][m] = f0;
                        acc[3][m] = f1;
                    } else {
                        acc[4][m] = f0;
                        acc[5][m] = f1;
                    }
                }
            }
            sb = sb + 1 == NBUF ? 0 : sb + 1;
        }
        // ---------------- forward lines
        // the unpacked outputs go to the stage buffer that no copy targets
        // until the next tile's first line (sb holds that line's inputs)
        cpx<float>* const H = stage0 + (sb ^ 1) * STG;
        for (int f = 0; f < NLO; ++f) {
            if constexpr (KIND == 0) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    if (f == 0) x[m] = mk(acc[0][m], acc[1][m]);
                    else if (f == 1) x[m] = mk(acc[2][m], acc[3][m]);
                    else x[m] = mk(acc[4][m], acc[5][m]);
                }
            } else {
                const float* eta = a.eta_src ? a.eta_src + (size_t)(r0 + c) * N + t : nullptr;
                switch (f) {
#define LDDMM_AF(F) \
    case F: adj_fields<F, E, TPL>(x, acc, S, eta, a.npts); break;
                    LDDMM_AF(0) LDDMM_AF(1) LDDMM_AF(2) LDDMM_AF(3) LDDMM_AF(4) LDDMM_AF(5)
                    LDDMM_AF(6) LDDMM_AF(7) LDDMM_AF(8) LDDMM_AF(9) LDDMM_AF(10) LDDMM_AF(11)
                    LDDMM_AF(12) LDDMM_AF(13) LDDMM_AF(14) LDDMM_AF(15) LDDMM_AF(16) LDDMM_AF(17)
#undef LDDMM_AF
                    default: break;
                }
                if (f + 1 < NLO) prefetch_line_fields<SS, N, TL>(tile_states, a.npts, (f + 1) / 6, (f + 1) % 6);
                if (f % 2 == 0) {
                    // (s, f_2): the two fields go to the line groups that
                    // transform them on row pairs (two rows of one field share
                    // a transform, as in the separate axis-2 pass); (f_0, f_1)
                    // of one group are alike in size and share this row's
                    // transform
                    float* const Ro = R + c * RP + t;
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        Ro[TPL * m] = x[m].x;
                        Ro[FS + TPL * m] = x[m].y;
                    }
                    __syncthreads();
                    const float* const Rq = R + q * FS + 2 * rp * RP + t;
#pragma unroll
                    for (int m = 0; m < E; ++m) x[m] = mk(Rq[TPL * m], Rq[RP + TPL * m]);
                }
            }
            fast_fft<float, N, 1, true, XA, true>(x, b0, b0, c, t, tws, -1);
            // every warp is done with the previous line's outputs in H
            __syncthreads();
            // unpack the two real rows' spectra: Z_k is register m of lane t
            // (k = t + TPL m); Z_{N-k} is register E - 1 - m of lane TPL - t
            // of the same line, or register (E - m) mod E of lane 0 itself
            // field-pair lines (tangent, adjoint (f_0, f_1)): H[0][row] and
            // H[1][row] are the two fields of the row; row-pair lines
            // (adjoint (s, f_2)): H[q][row] is field q of the line
            {
                const bool rowpair = KIND == 1 && f % 2 == 0;
                const int ha = rowpair ? q * TL + 2 * rp : c;
                const int hb = rowpair ? q * TL + 2 * rp + 1 : TL + c;
#pragma unroll
                for (int m = 0; m <= E / 2; ++m) {
                    if (TPL * m >= nb2) break;  // the same for every lane
                    const cpx<float> zn = partner_conj<float, E, TPL>(x, t, m);
                    const int k = t + TPL * m;
                    const cpx<float> zk = x[m];
                    if (k < nb2) {
                        H[ha * PH + k] = 0.5f * (zk + zn);
                        H[hb * PH + k] = rot(0.5f * (zk - zn), -1);
                    }
                }
            }
            __syncthreads();
            // outputs of this line: one combined F(s) + i kappa_2 F(f_2), or two plain
            const bool combined = KIND == 1 && (f % 2 == 0);
            int ob;
            if constexpr (KIND == 0) ob = 2 * f;
            else ob = 9 * (f / 6) + 3 * ((f % 6) / 2) + (combined ? 0 : 1);
            // thread -> (row, first plane): the TL rows of a plane are one
            // coalesced segment of the [k2][row] layout
            static_assert(FAST_THREADS % TL == 0, "whole planes per block sweep");
            const int orow = threadIdx.x % TL;
            constexpr int KSTEP = FAST_THREADS / TL;
            if (combined) {
                cpx<float>* const o = a.out[ob] + r0 + orow;
                for (int k = threadIdx.x / TL; k < nb2; k += KSTEP) {
                    const float d = dks[k];
                    const cpx<float> fs = H[orow * PH + k], f2 = H[(TL + orow) * PH + k];
                    o[(size_t)k * rows] = fs + mk(-d * f2.y, d * f2.x);
                }
            } else {
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                    cpx<float>* const o = a.out[ob + qq] + r0 + orow;
                    for (int k = threadIdx.x / TL; k < nb2; k += KSTEP)
                        o[(size_t)k * rows] = H[(qq * TL + orow) * PH + k];
                }
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace lddmm
