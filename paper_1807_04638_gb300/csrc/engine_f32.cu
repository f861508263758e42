// Single-precision engine (FP32 transport, shooting and K-apply; FP64 reductions).
#include "engine.cuh"

namespace lddmm {
EngineBase* make_engine_f32(const Dims& d, const lddmm_params& p, cudaStream_t s, lddmm_status* st) {
    Engine<float>* e = new Engine<float>(d, p, s);
    *st = e->init();
    return e;
}
}  // namespace lddmm
