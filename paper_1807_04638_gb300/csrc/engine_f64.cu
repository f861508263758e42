// Double-precision engine (the plain FP64 method).
#include "engine.cuh"

namespace lddmm {
EngineBase* make_engine_f64(const Dims& d, const lddmm_params& p, cudaStream_t s, lddmm_status* st) {
    Engine<double>* e = new Engine<double>(d, p, s);
    *st = e->init();
    return e;
}
}  // namespace lddmm
