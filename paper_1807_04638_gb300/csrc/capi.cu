// C ABI of liblddmm.so: argument checks, handle lifetime, dispatch to the
// double- or single-precision engine.  No C++ exception crosses this file.
#include <new>

#include "engine.cuh"

using namespace lddmm;

struct lddmm_handle {
    EngineBase* eng;
    int device;
};

static bool params_ok(const lddmm_params* p) {
    if (!p) return false;
    if (!(p->alpha > 0) || p->s < 1 || p->s > 8 || !(p->weight >= 0)) return false;
    if (p->nt < 1 || p->nt > 56) return false;
    if (p->interp != LDDMM_INTERP_CUBIC && p->interp != LDDMM_INTERP_LINEAR) return false;
    if (p->space != LDDMM_SPACE_V && p->space != LDDMM_SPACE_L2) return false;
    if (p->compute_dtype != LDDMM_F64 && p->compute_dtype != LDDMM_F32) return false;
    // stored states: the compute type, or bfloat16 with FP32 compute (precision form)
    if (p->state_dtype != p->compute_dtype && !(p->compute_dtype == LDDMM_F32 && p->state_dtype == LDDMM_BF16))
        return false;
    if (p->checkpoint_every < 1) return false;
    if (p->gn_maxit < 0 || p->pcg_maxit < 0 || p->ls_maxit < 1) return false;
    if (p->dealias != 0 && p->dealias != 1) return false;
    if (p->optimizer != LDDMM_OPT_GN && p->optimizer != LDDMM_OPT_GD) return false;
    if (p->gradient_mode != LDDMM_GRAD_JACOBI && p->gradient_mode != LDDMM_GRAD_DISCRETE) return false;
    // the transposed map steps read the stored stage velocities in the compute type
    if (p->gradient_mode == LDDMM_GRAD_DISCRETE && (p->state_dtype != p->compute_dtype || p->checkpoint_every > 1))
        return false;
    return true;
}

extern "C" {

void lddmm_default_params(lddmm_params* p) {
    if (!p) return;
    p->alpha = 0.01;
    p->s = 2;
    p->weight = 1e-3;
    p->nt = 10;
    p->interp = LDDMM_INTERP_CUBIC;
    p->space = LDDMM_SPACE_V;
    p->compute_dtype = LDDMM_F64;
    p->state_dtype = LDDMM_F64;
    p->checkpoint_every = 1;
    p->gn_maxit = 5;
    p->pcg_maxit = 10;
    p->pcg_rtol = 0.1;
    p->armijo_c1 = 1e-4;
    p->ls_maxit = 10;
    p->dealias = 1;
    p->optimizer = LDDMM_OPT_GN;
    p->gradient_mode = LDDMM_GRAD_JACOBI;
}

size_t lddmm_workspace_bytes(const lddmm_grid* g, const lddmm_params* p) {
    Dims d;
    if (!make_dims(g, &d) || !params_ok(p)) return 0;
    return layout_for(d, p, p->compute_dtype == LDDMM_F64 ? 8 : 4).bytes;
}

lddmm_status lddmm_create(lddmm_handle** h, const lddmm_grid* g, const lddmm_params* p, void* cuda_stream) {
    if (!h) return LDDMM_ERR_ARG;
    *h = nullptr;
    if (!params_ok(p)) return LDDMM_ERR_ARG;
    Dims d;
    if (!make_dims(g, &d)) return LDDMM_ERR_SHAPE;
    lddmm_handle* hh = new (std::nothrow) lddmm_handle;
    if (!hh) return LDDMM_ERR_OOM;
    if (cudaGetDevice(&hh->device) != cudaSuccess) {
        delete hh;
        return LDDMM_ERR_CUDA;
    }
    lddmm_status st = LDDMM_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    hh->eng = p->compute_dtype == LDDMM_F64 ? make_engine_f64(d, *p, s, &st) : make_engine_f32(d, *p, s, &st);
    if (!hh->eng || st != LDDMM_OK) {
        delete hh->eng;
        delete hh;
        return st != LDDMM_OK ? st : LDDMM_ERR_OOM;
    }
    *h = hh;
    return LDDMM_OK;
}

lddmm_status lddmm_destroy(lddmm_handle* h) {
    if (!h) return LDDMM_ERR_ARG;
    if (h->eng) h->eng->synchronize();
    delete h->eng;
    delete h;
    return LDDMM_OK;
}

const char* lddmm_status_string(lddmm_status s) {
    switch (s) {
        case LDDMM_OK: return "ok";
        case LDDMM_ERR_ARG: return "invalid argument";
        case LDDMM_ERR_SHAPE: return "unsupported grid shape (each axis must be 2..512 with factors 2, 3, 5)";
        case LDDMM_ERR_OOM: return "device out of memory";
        case LDDMM_ERR_CUDA: return "CUDA runtime error";
        case LDDMM_ERR_NOT_LINEARIZED: return "no linearisation point: call lddmm_gradient first";
        case LDDMM_ERR_NONFINITE: return "non-finite value in an input or a result";
        case LDDMM_ERR_DEVICE_CHECK: return "device-side or planner check failed";
        case LDDMM_ERR_TIMEOUT: return "host wait exceeded its limit";
        case LDDMM_WARN_LINESEARCH: return "Armijo line search failed; registration stopped early";
        case LDDMM_ERR_TOO_LARGE: return "grid too large for the fixed scratch of lddmm_apply_metric_noalloc";
    }
    return "unknown status";
}

lddmm_status lddmm_last_status(const lddmm_handle* h) { return h && h->eng ? h->eng->status : LDDMM_ERR_ARG; }

lddmm_status lddmm_synchronize(lddmm_handle* h) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->synchronize();
}

lddmm_status lddmm_shoot(lddmm_handle* h, const void* v0, const void* I0, void* m1, void* u1, double* kinetic) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->shoot(v0, I0, m1, u1, kinetic);
}

lddmm_status lddmm_gradient(lddmm_handle* h, const void* v0, const void* I0, const void* I1, void* grad,
                            double* energy) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->gradient(v0, I0, I1, grad, energy);
}

lddmm_status lddmm_hessvec(lddmm_handle* h, const void* dv0, void* Hdv) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->hessvec(dv0, Hdv);
}

lddmm_status lddmm_jacobi_forward(lddmm_handle* h, const void* dv0, void* eta1, void* xi1) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->jacobi_forward(dv0, eta1, xi1);
}

lddmm_status lddmm_jacobi_adjoint(lddmm_handle* h, const void* b_eta, const void* b_xi, void* out) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->jacobi_adjoint(b_eta, b_xi, out);
}

lddmm_status lddmm_apply_metric(lddmm_handle* h, const void* in, void* out, int ncomp, int power) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->apply_metric(in, out, ncomp, power);
}

lddmm_status lddmm_jacobian_det(lddmm_handle* h, const void* u, void* J, double* minmax) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->jacobian_det(u, J, minmax);
}

lddmm_status lddmm_shoot_vjp(lddmm_handle* h, const void* G, void* out) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->shoot_vjp(G, out);
}

lddmm_status lddmm_register(lddmm_handle* h, const void* I0, const void* I1, void* v0_inout, lddmm_report* report) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->reg(I0, I1, v0_inout, report);
}

int lddmm_profile_num_classes(void) { return KC_COUNT; }

const char* lddmm_profile_class_name(int cls) { return cls >= 0 && cls < KC_COUNT ? kclass_names[cls] : ""; }

lddmm_status lddmm_profile(lddmm_handle* h, int enable) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->profile(enable);
}

lddmm_status lddmm_profile_read(lddmm_handle* h, int cls, double* ms, double* bytes, long long* launches) {
    if (!h || !h->eng) return LDDMM_ERR_ARG;
    return h->eng->profile_read(cls, ms, bytes, launches);
}

}  // extern "C"
