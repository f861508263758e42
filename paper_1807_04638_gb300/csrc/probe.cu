// FP64 fused multiply-add rate probe (measurement; no counterpart in the
// paper).  The plain FP64 method runs its FFT butterflies on the FP64 units,
// whose rate on this part is far below its memory bandwidth per flop; this
// kernel measures that rate so that the FP64 path's roofline has a measured
// denominator.  Each thread runs PROBE_CHAINS independent dependent chains
// a <- fma(a, b, c) on runtime values (nothing folds at compile time) and
// stores their sum, so the work cannot be removed.
#include <cuda_runtime.h>

#include "lddmm.h"

namespace {
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fp64_fma(double* out, int iters) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const double b = 1.0 - 1e-9 * (double)(threadIdx.x & 7);
    const double c = 1e-12 * (double)tid;
    double a[PROBE_CHAINS];
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = 1.0 + 1e-3 * q + 1e-9 * tid;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = fma(a[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; ++q) s += a[q];
    out[tid] = s;
}
}  // namespace

extern "C" lddmm_status lddmm_probe_fp64_fma(double* out, int blocks, int iters, void* cuda_stream) {
    if (!out || blocks < 1 || iters < 1) return LDDMM_ERR_ARG;
    k_probe_fp64_fma<<<blocks, PROBE_THREADS, 0, (cudaStream_t)cuda_stream>>>(out, iters);
    return cudaGetLastError() == cudaSuccess ? LDDMM_OK : LDDMM_ERR_CUDA;
}

extern "C" double lddmm_probe_fp64_fma_flops(int blocks, int iters) {
    return 2.0 * PROBE_CHAINS * (double)iters * PROBE_THREADS * (double)blocks;
}

extern "C" int lddmm_probe_fp64_fma_threads(void) { return PROBE_THREADS; }
