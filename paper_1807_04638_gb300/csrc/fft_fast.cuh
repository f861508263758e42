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
//
// Band-limited transforms (PassParams::nb2, c1, s1): under the 2/3-rule
// projector P most of the half spectrum is zero or never used, so a pass can
// be restricted to the k2 planes and k1 columns of the band.  The axis-2 pass
// reads (inverse) or writes (forward) only the planes k2 < nb2; the axis-1
// pass transforms only the lines of those planes and reads (inverse) or
// writes (forward) only the band's k1 entries; the axis-0 pass transforms
// only the lines (k2, k1) inside the band.  Skipped inputs count as zero and
// skipped outputs are left unwritten.
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
// mixed radix: E is a multiple of every radix of the plan
template <> struct FastPlan<96> { static constexpr bool ok = true; static constexpr int E = 12, RADS = 0x3244; };
template <> struct FastPlan<192> { static constexpr bool ok = true; static constexpr int E = 12, RADS = 0x3444; };
template <> struct FastPlan<160> { static constexpr bool ok = true; static constexpr int E = 20, RADS = 0x5244; };

constexpr int FAST_THREADS = 256;
// Resident blocks per SM the register budget is sized for: 4 for FP32
// (<= 64 registers), 2 for FP64, so that enough loads are in flight to hide
// DRAM latency.
template <class T, int N> struct FastOcc {
    static constexpr int value = FastPlan<N>::E > 12 ? 1 : (sizeof(T) == 4 ? (FastPlan<N>::E > 8 ? 3 : 4) : 2);
};
// resident blocks of the persistent C2C passes (double-buffered tiles)
template <class T, int N> struct FastOccC2C {
    static constexpr int value = FastPlan<N>::E > 12 ? 1 : (FastPlan<N>::E > 8 ? 2 : 3);
};

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

// Shared-memory index of element p of line c.  A half-warp's 8-byte (FP32)
// or 16-byte (FP64) accesses are served together, so the layouts are chosen
// against a model of the 32 four-byte banks per half-warp, over every store
// and load of every Stockham exchange of the compiled plans:
//  MAP 0 (c fastest in a warp): odd line pitch (FP32, N = 256: one pad slot
//        every 8 elements and a pitch of N + N/8 + 2).
//  MAP 1 (t fastest in a warp): FP32, N = 128 / 192 / 256: the low four index
//        bits XOR-ed with a key linear in the higher bits (conflict-free, no
//        padding); otherwise one pad slot every 2^SH elements (conflict-free
//        except FP32 N = 96 and 160: 1.33 and 1.67 wavefronts per request).
template <class T, int N, int MAP> struct SIdx {
    static constexpr bool F32 = sizeof(T) == 4;
    static constexpr int KIND = MAP == 0 ? ((F32 && N == 256) ? 1 : 0)
                                         : ((F32 && (N == 128 || N == 192 || N == 256)) ? 2 : 1);
    static constexpr int SH = MAP == 0 ? 3
                                       : (F32 ? (N == 96 ? 4 : (N == 160 ? 2 : 3))
                                              : ((N == 128 || N == 256) ? 4 : 3));
    static constexpr int LP = KIND == 0 ? N + 1
                                        : (KIND == 2 ? N
                                                     : N + (N >> SH) + ((MAP == 0 || (F32 && N == 96)) ? 2 : 0));
    static __device__ __forceinline__ int swz(int p) {
        if constexpr (N == 128) {
            const int q = p >> 4;
            return p ^ ((q & 1) ^ (((q >> 1) & 1) * 10) ^ (q & 4));
        } else if constexpr (N == 256) {
            return p ^ ((p >> 3) & 15);
        } else {
            return p ^ ((p >> 2) & 15);
        }
    }
    static __device__ __forceinline__ int at(int c, int p) {
        if constexpr (KIND == 0) return c * LP + p;
        else if constexpr (KIND == 1) return c * LP + p + (p >> SH);
        else return c * LP + swz(p);
    }
};

// Barrier of a line's exchanges.  Only the TPL threads of a line touch its
// exchange tiles; with MAP 1 (t fastest) they are consecutive threads of one
// warp (TPL divides 32), so a warp barrier suffices, while with MAP 0 they
// are spread over the block.
template <int MAP, int TPL> __device__ __forceinline__ void line_sync() {
    if constexpr (MAP == 1) {
        static_assert(32 % TPL == 0, "a line's threads must lie in one warp");
        __syncwarp();
    } else {
        __syncthreads();
    }
}

// Per-stage twiddle tables in shared memory: stage S >= 1 (radix R, NS) keeps
// w^(k r N / (NS R)) at (r - 1) NS + k for k < NS, 1 <= r < R, so that the
// threads of a line read consecutive (or equal) entries: no bank conflicts.
template <int N, int S> struct StageTw {
    static constexpr int RADS = FastPlan<N>::RADS;
    static __host__ __device__ constexpr int radix(int s) { return (RADS >> (4 * s)) & 0xF; }
    static __host__ __device__ constexpr int ns(int s) { return s == 0 ? 1 : ns(s - 1) * radix(s - 1); }
    static __host__ __device__ constexpr int off(int s) {
        return s <= 1 ? 0 : off(s - 1) + (radix(s - 1) - 1) * ns(s - 1);
    }
    static constexpr int R = radix(S), NS = ns(S), OFF = off(S);
};
template <int N> struct TwTable {
    static __host__ __device__ constexpr int nstages() {
        int n = 0;
        for (int r = FastPlan<N>::RADS; r; r >>= 4) ++n;
        return n;
    }
    static constexpr int SIZE = StageTw<N, 15>::off(nstages());  // entries of all stages
};
// fill the per-stage tables from the twiddle table tw (e^{-2 pi i t / N}); all
// threads of the block call it
template <class T, int N>
__device__ __forceinline__ void fill_stage_twiddles(cpx<T>* tws, const cpx<T>* tw) {
    using ST = StageTw<N, 15>;
    constexpr int NST = TwTable<N>::nstages();
    for (int i = threadIdx.x; i < TwTable<N>::SIZE; i += blockDim.x) {
        int s = 1;
        while (s + 1 < NST && i >= ST::off(s + 1)) ++s;
        const int ns = ST::ns(s), R = ST::radix(s);
        const int j = i - ST::off(s), r = j / ns + 1, k = j % ns;
        tws[i] = ldg(tw + k * r * (N / (ns * R)));
    }
}

// Exchange addressing by XOR (XA).  With the XOR layout (SIdx KIND 2) and N
// a power of two, the element index of every exchange access splits into a
// thread part and a compile-time part with disjoint bits (radix digits of t,
// and of b, r or m), and the layout is linear over XOR: swz(P_t | P_c) =
// swz(P_t) ^ swz(P_c).  For a line whose shared-memory base is aligned to
// the line's size (8 N bytes) the byte address is therefore
// (base | 8 swz(P_t)) ^ 8 swz(P_c): one per-thread value per exchange, and
// one XOR with a constant per access.  The caller guarantees the alignment.
template <class T, int N> struct XorEx {
    static constexpr bool ok = sizeof(T) == 4 && SIdx<T, N, 1>::KIND == 2 && (N & (N - 1)) == 0;
    static __host__ __device__ constexpr int lg(int v) { return v <= 1 ? 0 : 1 + lg(v / 2); }
};
__device__ __forceinline__ void sts_v2(unsigned a, cpx<float> v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ cpx<float> lds_v2(unsigned a) {
    cpx<float> v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

// p advanced to the next ALIGN-byte boundary of the shared window (the
// kernel allocates ALIGN - 16 bytes more than it uses)
template <int ALIGN> __device__ __forceinline__ unsigned char* align_smem(unsigned char* p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    return p + ((ALIGN - (s & (ALIGN - 1))) & (ALIGN - 1));
}

// TWS: the twiddles are the per-stage tables in shared memory (else the
// global table, read through the read-only cache); XA: exchange addressing
// by XOR (MAP 1 lines of an XorEx<T, N>::ok plan on 8N-byte aligned tiles);
// ONEX: every exchange uses one tile (b1 == b0), and a stage waits for the
// line's loads of the previous exchange before it stores
template <class T, int N, int E, int TPL, int RADS, int S, int NS, int MAP, bool TWS = false, bool XA = false,
          bool ONEX = false>
__device__ __forceinline__ void fast_stages(cpx<T> (&x)[E], cpx<T>* b0, cpx<T>* b1, int c, int t, const cpx<T>* tw,
                                            int dir) {
    constexpr int R = (RADS >> (4 * S)) & 0xF;
    constexpr bool LAST = NS * R == N;
    constexpr int B = E / R;
    static_assert(B * R == E, "radix must divide the per-thread element count");
    static_assert(!XA || (MAP == 1 && XorEx<T, N>::ok), "XOR addressing needs the XOR layout of a power-of-two line");
    using SI = SIdx<T, N, MAP>;
    constexpr unsigned CB = (unsigned)sizeof(cpx<T>);
    if constexpr (ONEX && S > 0 && !LAST) line_sync<MAP, TPL>();
    // XA: this line's base in the shared window
    unsigned lb = 0;
    if constexpr (XA) lb = (unsigned)__cvta_generic_to_shared(b0) + (unsigned)(c * SI::LP) * CB;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + TPL * b;
        const int k = j % NS;
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cpx<T> a = x[b + B * r];
            if (NS > 1 && r > 0) {
                cpx<T> w = TWS ? tw[StageTw<N, S>::OFF + (r - 1) * NS + k] : ldg(&tw[k * r * (N / (NS * R))]);
                if (dir > 0) w.y = -w.y;
                a = a * w;
            }
            v[r] = a;
        }
        dft_r<T, R>(v, dir);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[b + B * r] = v[r];
        } else if constexpr (XA) {
            // store index (j / NS) NS R + k + r NS: thread part from t, the
            // rest from b and r
            constexpr int LNS = XorEx<T, N>::lg(NS), LR = XorEx<T, N>::lg(R);
            const int pt = ((t >> LNS) << (LNS + LR)) | (t & (NS - 1));
            const unsigned as = lb | CB * (unsigned)SI::swz(pt);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int pc = (((TPL * b) >> LNS) << (LNS + LR)) | ((TPL * b) & (NS - 1)) | (r << LNS);
                sts_v2(as ^ CB * (unsigned)SI::swz(pc), v[r]);
            }
        } else {
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) b0[SI::at(c, base + r * NS)] = v[r];
        }
    }
    if constexpr (!LAST) {
        line_sync<MAP, TPL>();
        if constexpr (XA) {
            // load index t + TPL m
            const unsigned al = lb | CB * (unsigned)SI::swz(t);
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = lds_v2(al ^ CB * (unsigned)SI::swz(TPL * m));
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = b0[SI::at(c, t + TPL * m)];
        }
        fast_stages<T, N, E, TPL, RADS, S + 1, NS * R, MAP, TWS, XA, ONEX>(x, b1, b0, c, t, tw, dir);
    }
}

template <class T, int N, int MAP, bool TWS = false, bool XA = false, bool ONEX = false>
__device__ __forceinline__ void fast_fft(cpx<T> (&x)[FastPlan<N>::E], cpx<T>* b0, cpx<T>* b1, int c, int t,
                                         const cpx<T>* tw, int dir) {
    constexpr int E = FastPlan<N>::E;
    line_sync<MAP, N / E>();  // the line's tiles may still be read by its previous transform
    fast_stages<T, N, E, N / E, FastPlan<N>::RADS, 0, 1, MAP, TWS, XA, ONEX>(x, b0, b1, c, t, tw, dir);
}

// conj(Z_{N-k}) for element k = t + TPL m of a line transform held as the
// register-blocked passes leave it (element t + TPL m in register m of lane
// t of the line's TPL consecutive lanes): register E - 1 - m of lane TPL - t,
// or register (E - m) mod E of lane 0 itself.  Every lane of the warp must
// call it (warp shuffles); m must be a compile-time index after unrolling.
template <class T, int E, int TPL>
__device__ __forceinline__ cpx<T> partner_conj(const cpx<T> (&x)[E], int t, int m) {
    const int lane = threadIdx.x & 31;
    const int src = (lane & ~(TPL - 1)) | ((TPL - t) & (TPL - 1));
    const T px = __shfl_sync(0xffffffffu, x[E - 1 - m].x, src);
    const T py = __shfl_sync(0xffffffffu, x[E - 1 - m].y, src);
    return t == 0 ? cj(x[(E - m) % E]) : mk(px, -py);
}

// ---------------------------------------------------------------- async copies
// 16-byte asynchronous global -> shared copies (cp.async, completion by
// commit / wait groups: no polling loop).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int P> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(P) : "memory");
}

// sym_apply over the E elements a thread holds of a line along axis AX
// (element m has index p = t + TPL m on that axis), in place.  The branches
// on the symbol's fields and the fixed axes' table entries are taken once per
// line, not per element; the line axis' kappa^2 and derivative tables are
// read from shared memory (ksqs, dks).  Every element gets sym_apply's
// arithmetic in sym_apply's order.
// kf0, kf1: the indices of the two fixed axes (k0 or k1, then k2).
template <class T, int AX, int E, int TPL>
__device__ __forceinline__ void sym_line(const SymT<T>& sy, const SpecTabs<T>& tb, const T* ksqs, const T* dks,
                                         int kf0, int k2, int t, cpx<T> (&v)[E]) {
    constexpr int AO = AX == 0 ? 1 : 0;  // the other in-plane axis (fixed along the line)
    if (sy.mask) {
        // fixed axes outside the band: the whole line is zero
        const bool outl = (kf0 > tb.kcut[AO] && kf0 < tb.n[AO] - tb.kcut[AO]) || k2 > tb.kcut[2];
        if (outl) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = mk((T)0, (T)0);
            return;
        }
    }
    T f[E];
    if (sy.lpow != 0) {
        const T qo = tb.ksq[AO][kf0], q2 = tb.ksq[2][k2];
        T base[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const T qa = ksqs[t + TPL * m];
            base[m] = (T)1 + tb.alpha * ((AX == 0 ? qa + qo : qo + qa) + q2);
        }
        const int e = tb.s * (sy.lpow > 0 ? sy.lpow : -sy.lpow);
        if (e == 2) {
#pragma unroll
            for (int m = 0; m < E; ++m) base[m] = base[m] * base[m];
        } else if (e == 4) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const T b2 = base[m] * base[m];
                base[m] = b2 * b2;
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                T pw = (T)1;
                for (int q = 0; q < e; ++q) pw *= base[m];
                base[m] = pw;
            }
        }
        if (sy.lpow > 0) {
#pragma unroll
            for (int m = 0; m < E; ++m) f[m] = sy.scale * base[m];
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) f[m] = sym_div(sy.scale, base[m]);
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) f[m] = sy.scale;
    }
    if (sy.deriv >= 0) {
        if (sy.deriv == AX) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const T d = dks[t + TPL * m] * f[m];
                v[m] = mk(-d * v[m].y, d * v[m].x);
            }
        } else {
            const T dk = tb.dk[sy.deriv][sy.deriv == 2 ? k2 : kf0];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const T d = dk * f[m];
                v[m] = mk(-d * v[m].y, d * v[m].x);
            }
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = mk(f[m] * v[m].x, f[m] * v[m].y);
    }
    if (sy.mask) {
        // line-axis entries outside the band
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int p = t + TPL * m;
            if (p > tb.kcut[AX] && p < tb.n[AX] - tb.kcut[AX]) v[m] = mk((T)0, (T)0);
        }
    }
}

// ---------------------------------------------------------------- C2C passes
// Persistent blocks walk the (tile, job) work items of the launch; every
// input tile of an item is a "load unit".  The next unit is copied into the
// other half of a double-buffered shared-memory tile (cp.async) while the
// current one is transformed, so DRAM latency overlaps the butterflies.
//   AXIS 1: a tile is TL consecutive contiguous lines along k1 ([line][N]).
//   AXIS 0: a tile is TL consecutive k1 columns of lines along k0 ([row][TL]).
//   Exchange tiles: axis 1 (its line's threads in one warp) uses one tile for
//   every exchange.  Axis 0 alternates between two tiles (exchange j in
//   tile j mod 2); with an odd number of stages (3, 5, ...) the last exchange
//   is in tile 1, so every read of tile 0 ends before the block barrier of a
//   later exchange, and tile 0 can be the stage buffer of the unit being
//   transformed (its tile is in registers by then): no copy refills it
//   before that barrier.  The rest of the SM's storage stays L1 for the bases.
template <class T, int N, int AXIS> struct C2CGeom {
    static constexpr int E = FastPlan<N>::E;
    static constexpr int TPL = N / E;
    static constexpr int TL = FAST_THREADS / TPL;
    static constexpr int MAP = AXIS == 1 ? 1 : 0;
    static constexpr int TILE = TL * N;  // complex elements of one staged tile
    static constexpr int XT = TL * SIdx<T, N, MAP>::LP;  // one exchange tile
    static constexpr bool ALIAS = AXIS == 0 && TwTable<N>::nstages() >= 3 && TwTable<N>::nstages() % 2 == 1;
    static constexpr int SB = ALIAS && XT > TILE ? XT : TILE;  // one stage buffer
    static constexpr size_t smem() {
        return ((size_t)2 * SB + (size_t)(AXIS == 1 || ALIAS ? 1 : 2) * XT + (size_t)N) * sizeof(cpx<T>) +
               (size_t)2 * N * sizeof(T);  // + twiddles, kappa^2 and derivative tables of the axis
    }
};

template <class T, int N, int AXIS>
__global__ void __launch_bounds__(FAST_THREADS, (FastOccC2C<T, N>::value)) k_fast_c2c(const __grid_constant__ PassParams<T> pp, int ntiles) {
    using G = C2CGeom<T, N, AXIS>;
    constexpr int E = G::E, TPL = G::TPL, TL = G::TL, MAP = G::MAP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the two stage buffers: stage0 + sb * SB (pointer arithmetic, not an
    // indexed array, which would live in local memory)
    cpx<T>* const stage0 = (cpx<T>*)smem_raw;
    cpx<T>* const xt = stage0 + 2 * G::SB;  // exchange tile(s)
    // the axis' twiddles and symbol tables in shared memory (the first
    // barrier of the main loop orders these stores before their reads)
    cpx<T>* const tws = xt + (AXIS == 1 || G::ALIAS ? 1 : 2) * G::XT;
    T* const ksqs = (T*)(tws + N);
    T* const dks = ksqs + N;
    static_assert(TwTable<N>::SIZE <= N, "per-stage twiddle tables fit N entries");
    fill_stage_twiddles<T, N>(tws, (const cpx<T>*)pp.ax.tw);
    for (int i = threadIdx.x; i < N; i += FAST_THREADS) {
        ksqs[i] = pp.tabs.ksq[AXIS][i];
        dks[i] = pp.tabs.dk[AXIS][i];
    }
    const int n0 = pp.n0, n1 = pp.n1, n2h = pp.n2h;
    const int nitems = ntiles * pp.njobs;
    int c, t;
    if (MAP == 1) {
        c = threadIdx.x / TPL;
        t = threadIdx.x % TPL;
    } else {
        c = threadIdx.x % TL;
        t = threadIdx.x / TL;
    }
    // band: k2 planes < nb2; k1 columns [0, c1) and [s1, n1)
    const int nb2 = pp.nb2, c1 = pp.c1, s1 = pp.s1;
    const int tA = (c1 + TL - 1) / TL;                // AXIS 0: tiles of the first column range
    const int tpk = tA + (n1 - s1 + TL - 1) / TL;      // AXIS 0: tiles per k2 plane
    (void)n2h;

    // geometry of a tile: first global element, valid lines (columns)
    auto tile_geo = [&](int tile, int& g0, int& nval, int& k2t, int& kb) {
        if (AXIS == 1) {
            const int line0 = tile * TL;
            nval = min(TL, nb2 * n0 - line0);
            g0 = line0 * n1;
            k2t = 0;
            kb = line0;
        } else {
            k2t = (int)pp.fd_tpk.div((unsigned)tile);
            const int r = tile - k2t * tpk;
            if (r < tA) {
                kb = r * TL;
                nval = min(TL, c1 - kb);
            } else {
                kb = s1 + (r - tA) * TL;
                nval = min(TL, n1 - kb);
            }
            g0 = k2t * n0 * n1 + kb;
        }
    };
    // AXIS 1 inverse: spectral entries k1 in [c1, s1) are zero (not read)
    auto k1_out = [&](int p) { return AXIS == 1 && p >= c1 && p < s1; };
    // issue the copy of input q of item w into stage buffer sb
    // work item w -> (job, tile)
    auto split = [&](int w, int& jw, int& tile) {
        jw = (int)pp.fd_tiles.div((unsigned)w);
        tile = w - jw * ntiles;
    };
    auto issue = [&](int w, int q, int sb) {
        if (w < nitems) {
            int jw, tl;
            split(w, jw, tl);
            const PassJobT<T>& jb = pp.jobs[jw];
            const cpx<T>* src = (const cpx<T>*)jb.in[q];
            int g0, nval, k2t, kb;
            tile_geo(tl, g0, nval, k2t, kb);
            if (AXIS == 1) {
                const int chunks = nval * N * (int)sizeof(cpx<T>) / 16;
                const bool skip = pp.sign > 0 && c1 < s1;
                for (int i = threadIdx.x; i < chunks; i += FAST_THREADS) {
                    // c1, s1 are even: a 16-byte chunk lies wholly inside or outside the band
                    if (skip && k1_out((16 * i / (int)sizeof(cpx<T>)) % N)) continue;
                    cp_async16((char*)(stage0 + sb * G::SB) + 16 * i, (const char*)(src + g0) + 16 * i);
                }
            } else {
                // 16-byte chunks per row: CPR for a full tile (compile time), cpr valid
                constexpr int CPR = TL * (int)sizeof(cpx<T>) / 16;
                const int cpr = nval * (int)sizeof(cpx<T>) / 16;
                for (int i = threadIdx.x; i < N * CPR; i += FAST_THREADS) {
                    const int p = i / CPR, ch = i % CPR;
                    if (ch < cpr)
                        cp_async16((char*)((stage0 + sb * G::SB) + p * TL) + 16 * ch,
                                   (const char*)(src + g0 + p * n1) + 16 * ch);
                }
            }
        }
        cp_async_commit();
    };

    // the unit sequence: items w = blockIdx.x, +gridDim.x, ...; inputs q = 0..nin-1
    int w = blockIdx.x, q = 0, sb = 0;
    int nw = w, nq = 0;  // the unit being prefetched
    auto advance = [&](int& ww, int& qq) {
        const PassJobT<T>& jb = pp.jobs[pp.fd_tiles.div((unsigned)ww)];
        if (++qq >= jb.nin) {
            qq = 0;
            ww += gridDim.x;
        }
    };
    if (w < nitems) issue(nw, nq, 0);
    advance(nw, nq);
    cpx<T> x[E], acc[E];
    while (w < nitems) {
        // prefetch the next unit into the other buffer, then wait for this one
        if (nw < nitems) issue(nw, nq, sb ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        int jw, tl;
        split(w, jw, tl);
        const PassJobT<T>& job = pp.jobs[jw];
        int g0, nval, k2t, kb;
        tile_geo(tl, g0, nval, k2t, kb);
        const bool valid = c < nval;
        const cpx<T>* tile = (stage0 + sb * G::SB);
        // this unit's exchange tiles
        cpx<T>* const b0 = AXIS == 1 ? xt : (G::ALIAS ? stage0 + sb * G::SB : xt);
        cpx<T>* const b1 = AXIS == 1 ? xt : (G::ALIAS ? xt : xt + G::XT);
        // frequency indices of the other two axes for this thread's line
        int k0b, k1b, k2b;
        if (AXIS == 1) {
            const int line = kb + (valid ? c : 0);
            k2b = (int)pp.fd_n0.div((unsigned)line);
            k0b = line - k2b * n0;
            k1b = 0;
        } else {
            k2b = k2t;
            k1b = kb + (valid ? c : 0);
            k0b = 0;
        }
        auto at = [&](int p) { return AXIS == 1 ? c * N + p : p * TL + c; };
        auto gidx = [&](int p) { return AXIS == 1 ? g0 + c * n1 + p : g0 + p * n1 + c; };
        const bool last = q == job.nin - 1;
        if (pp.sign > 0) {
            // inverse: lincomb of the inputs, then each output's symbol, IFFT, store
            const T coef = job.isym[q].scale;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int p = t + TPL * m;
                const cpx<T> v = valid && !k1_out(p) ? tile[at(p)] : mk((T)0, (T)0);
                acc[m] = q == 0 ? coef * v : acc[m] + coef * v;
            }
            __syncthreads();  // the stage buffer may now be refilled
            if (last) {
                for (int o = 0; o < job.nout; ++o) {
                    const SymT<T> sy = job.osym[o];
#pragma unroll
                    for (int m = 0; m < E; ++m) x[m] = acc[m];
                    sym_line<T, AXIS, E, TPL>(sy, pp.tabs, ksqs, dks, AXIS == 0 ? k1b : k0b, k2b, t, x);
                    fast_fft<T, N, MAP, true, false, AXIS == 1>(x, b0, b1, c, t, tws, +1);
                    if (valid) {
                        cpx<T>* ob = (cpx<T>*)job.out[o] + gidx(t);
                        const int sm = AXIS == 1 ? TPL : TPL * n1;  // element step between m
#pragma unroll
                        for (int m = 0; m < E; ++m) ob[m * sm] = x[m];
                    }
                }
            }
        } else {
            // forward: FFT of each input, post-symbol, accumulate; bases and store after the last
            if (last && valid) {
                // the bases are read after the transform: bring them into L1 now
                const int g0t = gidx(t);
                const int sm = AXIS == 1 ? TPL : TPL * n1;
                for (int b = 0; b < job.nb; ++b) {
                    const cpx<T>* bp = (const cpx<T>*)job.base[b] + g0t;
#pragma unroll
                    for (int m = 0; m < E; ++m) asm volatile("prefetch.global.L1 [%0];" ::"l"(bp + m * sm));
                }
            }
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = valid ? tile[at(t + TPL * m)] : mk((T)0, (T)0);
            __syncthreads();
            fast_fft<T, N, MAP, true, false, AXIS == 1>(x, b0, b1, c, t, tws, -1);
            const SymT<T> sy = job.isym[q];
sym_line<T, AXIS, E, TPL>(sy, pp.tabs, ksqs, dks, AXIS == 0 ? k1b : k0b, k2b, t, x);
#pragma unroll
            for (int m = 0; m < E; ++m) acc[m] = q == 0 ? x[m] : acc[m] + x[m];
            if (last && valid) {
                const int g0t = gidx(t);
                const int sm = AXIS == 1 ? TPL : TPL * n1;  // element step between m
                for (int b = 0; b < job.nb; ++b) {
                    const cpx<T>* bp = (const cpx<T>*)job.base[b] + g0t;
                    const T bc = job.bcoef[b];
#pragma unroll
                    for (int m = 0; m < E; ++m)
                        if (!k1_out(t + TPL * m)) acc[m] = acc[m] + bc * bp[m * sm];
                }
                cpx<T>* ob = (cpx<T>*)job.out[0] + g0t;
#pragma unroll
                for (int m = 0; m < E; ++m)
                    if (!k1_out(t + TPL * m)) ob[m * sm] = acc[m];  // outside the band: not written
            }
        }
        // next unit
        w = nw;
        q = nq;
        if (nw < nitems) advance(nw, nq);
        sb ^= 1;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- axis-2 pass
// A block owns 2*TL consecutive rows, packed as TL complex lines; the half
// spectrum of the block is staged in H[row][k] (pitch Ph) for the transposed
// [k2][row] spectral layout.
template <class T, int N>
__global__ void __launch_bounds__(FAST_THREADS, (FastOcc<T, N>::value)) k_fast_axis2(const __grid_constant__ PassParams<T> pp) {
    constexpr int E = FastPlan<N>::E;
    constexpr int TPL = N / E;
    constexpr int TL = FAST_THREADS / TPL;
    constexpr int NH = N / 2 + 1;
    constexpr int PH = (NH % 2 == 0) ? NH + 1 : NH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* H = (cpx<T>*)smem_raw;
    cpx<T>* b0 = H + 2 * TL * PH;
    cpx<T>* b1 = b0 + TL * SIdx<T, N, 1>::LP;
    const PassJobT<T>& job = pp.jobs[blockIdx.y];
    const cpx<T>* tw = (const cpx<T>*)pp.ax.tw;
    const int rows = pp.n0 * pp.n1;
    const int r0 = blockIdx.x * 2 * TL;
    const int nr = min(2 * TL, rows - r0);
    const int c = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const bool va = 2 * c < nr, vb = 2 * c + 1 < nr;
    cpx<T> x[E];
    // staging geometry: thread -> (row of the block, first k), KS k per sweep
    static_assert(FAST_THREADS % (2 * TL) == 0, "rows of a block must tile the threads");
    constexpr int KS = FAST_THREADS / (2 * TL);
    const int srow = threadIdx.x % (2 * TL), sk = threadIdx.x / (2 * TL);
    const bool rv = srow < nr;
    const int nb2 = pp.nb2;
    if (pp.sign > 0) {
        // H[row][k] = sum_b c_b in_b[k][r0 + row] on the band, zero above it
        if (job.nin == 1) {
            const cpx<T>* src = (const cpx<T>*)job.in[0] + (r0 + srow);
            const T c0 = job.isym[0].scale;
            for (int k = sk; k < NH; k += KS)
                H[srow * PH + k] = rv && k < nb2 ? c0 * src[k * rows] : mk((T)0, (T)0);
        } else {
            for (int k = sk; k < NH; k += KS) {
                cpx<T> acc = mk((T)0, (T)0);
                if (rv && k < nb2)
                    for (int b = 0; b < job.nin; ++b)
                        acc = acc + job.isym[b].scale * ((const cpx<T>*)job.in[b])[k * rows + r0 + srow];
                H[srow * PH + k] = acc;
            }
        }
        for (int o = 0; o < job.nout; ++o) {
            const SymT<T> sy = job.osym[o];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = t + TPL * m;
                const bool lo = k < NH;
                const int kk = lo ? k : N - k;
                cpx<T> a, b;
                if constexpr (sizeof(T) == 4) {
                    const cpx<T> sc = sym_coef(sy, pp.tabs, 0, 0, kk);  // same for both rows
                    a = sym_mul(sc, H[(2 * c) * PH + kk]);
                    b = sym_mul(sc, H[(2 * c + 1) * PH + kk]);
                } else {  // FP64 is bound by its multiplies: apply the symbol directly
                    a = sym_apply(sy, pp.tabs, 0, 0, kk, H[(2 * c) * PH + kk]);
                    b = sym_apply(sy, pp.tabs, 0, 0, kk, H[(2 * c + 1) * PH + kk]);
                }
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
            T* oa = (T*)job.out[o] + ((r0 + 2 * c) * N + t);  // row pair (2c, 2c + 1)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                if (va) oa[TPL * m] = x[m].x;
                if (vb) oa[N + TPL * m] = x[m].y;
            }
        }
    } else {
        for (int q = 0; q < job.nin; ++q) {
            const T* ia = (const T*)job.in[q] + ((r0 + 2 * c) * N + t);  // row pair (2c, 2c + 1)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const T a = va ? ia[TPL * m] : (T)0;
                const T b = vb ? ia[N + TPL * m] : (T)0;
                x[m] = mk(a, b);
            }
            fast_fft<T, N, 1>(x, b0, b1, c, t, tw, -1);
            // pair Z_k with Z_{N-k} (warp shuffles; the H rows are this line's)
            const SymT<T> sy = job.isym[q];
#pragma unroll
            for (int m = 0; m <= E / 2; ++m) {
                if (TPL * m >= nb2) break;  // the same for every lane
                const cpx<T> zn = partner_conj<T, E, TPL>(x, t, m);
                const cpx<T> zk = x[m];
                const int k = t + TPL * m;
                if (k >= nb2) continue;
                cpx<T> sa, sb;
                if constexpr (sizeof(T) == 4) {
                    const cpx<T> sc = sym_coef(sy, pp.tabs, 0, 0, k);  // same for both rows
                    sa = sym_mul(sc, (T)0.5 * (zk + zn));
                    sb = sym_mul(sc, rot((T)0.5 * (zk - zn), -1));
                } else {
                    sa = sym_apply(sy, pp.tabs, 0, 0, k, (T)0.5 * (zk + zn));
                    sb = sym_apply(sy, pp.tabs, 0, 0, k, rot((T)0.5 * (zk - zn), -1));
                }
                cpx<T>* ha = &H[(2 * c) * PH + k];
                cpx<T>* hb = &H[(2 * c + 1) * PH + k];
                *ha = q == 0 ? sa : *ha + sa;
                *hb = q == 0 ? sb : *hb + sb;
            }
        }
        __syncthreads();
        cpx<T>* dst = (cpx<T>*)job.out[0] + (r0 + srow);
        if (rv)
            for (int k = sk; k < nb2; k += KS) dst[k * rows] = H[srow * PH + k];
    }
}

// ---------------------------------------------------------------- axis-2 pass, persistent
// The transforms of k_fast_axis2 for FP32 grids whose row count is a multiple
// of the tile (2*TL rows) and whose inverse jobs have one input.  Persistent
// blocks walk the (tile, job) work items; the next unit's input is staged with
// cp.async into the other half of a double buffer while the current one is
// transformed:
//   inverse: the band planes k2 < nb2 of the tile's rows, S[k][row] with a
//            16-byte pitch SP, read back as row pairs;
//   forward: the tile's 2*TL real rows of one input (contiguous), one unit
//            per input of the job.
template <class T, int N> struct A2Geom {
    static constexpr int E = FastPlan<N>::E;
    static constexpr int TPL = N / E;
    static constexpr int TL = FAST_THREADS / TPL;
    static constexpr int R2 = 2 * TL;                          // rows per tile
    static constexpr int NH = N / 2 + 1;
    static constexpr int PH = (NH % 2 == 0) ? NH + 1 : NH;     // H pitch (forward)
    static constexpr int SP = R2 + 16 / (int)sizeof(cpx<T>);   // inverse stage pitch
    static constexpr int SI = NH * SP;                         // inverse stage (complex)
    static constexpr int SF = R2 * N / 2;                      // forward stage (complex)
    static constexpr int XT = TL * SIdx<T, N, 1>::LP;          // one exchange tile
    static constexpr int SS0 = SI > SF ? SI : SF;
    static constexpr int SS = SS0 > XT ? SS0 : XT;             // one stage buffer (also an exchange tile)
    static constexpr int HS = R2 * PH > XT ? R2 * PH : XT;     // H (forward) / b0 (inverse)
    static constexpr int CPK = R2 * (int)sizeof(cpx<T>) / 16;  // 16-byte chunks per plane
    static constexpr int CPF = R2 * N * (int)sizeof(T) / 16;   // 16-byte chunks per input
};

constexpr int A2P_BLOCKS = 3;  // resident blocks per SM of the persistent axis-2 pass

template <class T, int N>
__global__ void __launch_bounds__(FAST_THREADS, A2P_BLOCKS) k_fast_axis2p(const __grid_constant__ PassParams<T> pp, int ntiles) {
    using G = A2Geom<T, N>;
    constexpr int E = G::E, TPL = G::TPL, TL = G::TL, R2 = G::R2, NH = G::NH, PH = G::PH, SP = G::SP;
    static_assert(FAST_THREADS % R2 == 0, "rows of a tile must tile the threads");
    constexpr int KS = FAST_THREADS / R2;
    static_assert(TL * SIdx<T, N, 1>::LP <= G::SS, "an exchange tile must fit a stage buffer");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* const stage0 = (cpx<T>*)smem_raw;  // buffers stage0 + sb * SS
    cpx<T>* const H = stage0 + 2 * G::SS;      // HS elements: forward H, or the inverse's b0
    cpx<T>* const b1 = H + G::HS;
    const cpx<T>* tw = (const cpx<T>*)pp.ax.tw;
    const int rows = pp.n0 * pp.n1;
    const int nb2 = pp.nb2;
    const int nitems = ntiles * pp.njobs;
    const bool inv = pp.sign > 0;
    const int c = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int srow = threadIdx.x % R2, sk = threadIdx.x / R2;

    auto split = [&](int w, int& jw, int& tile) {
        jw = (int)pp.fd_tiles.div((unsigned)w);
        tile = w - jw * ntiles;
    };
    auto issue = [&](int w, int q, int sb) {
        if (w < nitems) {
            int jw, tl;
            split(w, jw, tl);
            const PassJobT<T>& jb = pp.jobs[jw];
            const int r0 = tl * R2;
            cpx<T>* dst = stage0 + sb * G::SS;
            if (inv) {
                const cpx<T>* src = (const cpx<T>*)jb.in[0] + r0;
                for (int i = threadIdx.x; i < nb2 * G::CPK; i += FAST_THREADS) {
                    const int k = i / G::CPK, ch = i % G::CPK;
                    cp_async16((char*)(dst + k * SP) + 16 * ch, (const char*)(src + k * rows) + 16 * ch);
                }
            } else {
                const char* src = (const char*)((const T*)jb.in[q] + r0 * N);
                for (int i = threadIdx.x; i < G::CPF; i += FAST_THREADS)
                    cp_async16((char*)dst + 16 * i, src + 16 * i);
            }
        }
        cp_async_commit();
    };
    // units: one per item (inverse) or one per input of the item's job (forward)
    auto advance = [&](int& ww, int& qq) {
        if (inv || ++qq >= pp.jobs[pp.fd_tiles.div((unsigned)ww)].nin) {
            qq = 0;
            ww += gridDim.x;
        }
    };
    int w = blockIdx.x, q = 0, sb = 0;
    int nw = w, nq = 0;
    if (w < nitems) {
        issue(nw, nq, 0);
        advance(nw, nq);
    }
    cpx<T> x[E];
    while (w < nitems) {
        if (nw < nitems) issue(nw, nq, sb ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        int jw, tl;
        split(w, jw, tl);
        const PassJobT<T>& job = pp.jobs[jw];
        const int r0 = tl * R2;
        cpx<T>* const S = stage0 + sb * G::SS;
        // first exchange tile: the inverse reads its staged planes for every
        // output, so it uses the H region (unused by the inverse); the forward
        // reads its stage buffer into registers before transforming, so the
        // buffer itself serves
        cpx<T>* const b0 = inv ? H : S;
        if (inv) {
            const T c0 = job.isym[0].scale;
            for (int o = 0; o < job.nout; ++o) {
                const SymT<T> sy = job.osym[o];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int k = t + TPL * m;
                    const bool lo = k < NH;
                    const int kk = lo ? k : N - k;
                    cpx<T> a = mk((T)0, (T)0), b = mk((T)0, (T)0);
                    if (kk < nb2) {  // planes above the band are zero (not staged)
                        const cpx<T>* pr = S + kk * SP + 2 * c;
                        a = c0 * pr[0];
                        b = c0 * pr[1];
                    }
                    const cpx<T> sc = sym_coef(sy, pp.tabs, 0, 0, kk);
                    a = sym_mul(sc, a);
                    b = sym_mul(sc, b);
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
                T* oa = (T*)job.out[o] + ((r0 + 2 * c) * N + t);  // row pair (2c, 2c + 1)
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    oa[TPL * m] = x[m].x;
                    oa[N + TPL * m] = x[m].y;
                }
            }
        } else {
            const T* Sr = (const T*)S + (2 * c) * N + t;  // row pair (2c, 2c + 1) of the tile
#pragma unroll
            for (int m = 0; m < E; ++m) x[m] = mk(Sr[TPL * m], Sr[N + TPL * m]);
            // the exchange tile is the stage buffer itself: with a padded line
            // pitch a line's exchange region overlaps the next line's rows, so
            // every line must have read its rows first
            if constexpr (SIdx<T, N, 1>::LP != N) __syncthreads();
            fast_fft<T, N, 1>(x, b0, b1, c, t, tw, -1);
            // pair Z_k with Z_{N-k} (warp shuffles; the H rows are this line's)
            const SymT<T> sy = job.isym[q];
#pragma unroll
            for (int m = 0; m <= E / 2; ++m) {
                if (TPL * m >= nb2) break;  // the same for every lane
                const cpx<T> zn = partner_conj<T, E, TPL>(x, t, m);
                const cpx<T> zk = x[m];
                const int k = t + TPL * m;
                if (k >= nb2) continue;
                const cpx<T> sc = sym_coef(sy, pp.tabs, 0, 0, k);
                const cpx<T> sa = sym_mul(sc, (T)0.5 * (zk + zn));
                const cpx<T> sbv = sym_mul(sc, rot((T)0.5 * (zk - zn), -1));
                cpx<T>* ha = &H[(2 * c) * PH + k];
                cpx<T>* hb = &H[(2 * c + 1) * PH + k];
                *ha = q == 0 ? sa : *ha + sa;
                *hb = q == 0 ? sbv : *hb + sbv;
            }
            if (q == job.nin - 1) {
                __syncthreads();
                cpx<T>* dst = (cpx<T>*)job.out[0] + (r0 + srow);
                for (int k = sk; k < nb2; k += KS) dst[k * rows] = H[srow * PH + k];
            }
        }
        __syncthreads();  // the stage buffer and H may now be refilled
        w = nw;
        q = nq;
        if (nw < nitems) advance(nw, nq);
        sb ^= 1;
    }
    cp_async_wait<0>();
}

template <class T, int N> constexpr size_t fast_axis2p_smem() {
    using G = A2Geom<T, N>;
    return ((size_t)2 * G::SS + (size_t)G::HS + (size_t)G::XT) * sizeof(cpx<T>);
}

template <class T, int N> constexpr size_t fast_c2c_smem(int axis) {
    return axis == 1 ? C2CGeom<T, N, 1>::smem() : C2CGeom<T, N, 0>::smem();
}
template <class T, int N> constexpr size_t fast_axis2_smem() {
    constexpr int TL = FAST_THREADS / (N / FastPlan<N>::E);
    constexpr int NH = N / 2 + 1;
    constexpr int PH = (NH % 2 == 0) ? NH + 1 : NH;
    return ((size_t)2 * TL * PH + (size_t)2 * TL * SIdx<T, N, 1>::LP) * sizeof(cpx<T>);
}

}  // namespace lddmm
