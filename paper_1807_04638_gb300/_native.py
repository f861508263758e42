"""ctypes binding of liblddmm.so (argument marshalling only).

Every numerical step runs in the CUDA library; this module converts torch
tensors to device pointers and the library's status codes to exceptions.
There is no fallback: if the library is missing, importing the binding
raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "liblddmm.so")

LDDMM_F64, LDDMM_F32, LDDMM_BF16 = 0, 1, 2
LDDMM_INTERP_CUBIC, LDDMM_INTERP_LINEAR = 0, 1
LDDMM_SPACE_V, LDDMM_SPACE_L2 = 0, 1
LDDMM_OPT_GN, LDDMM_OPT_GD = 0, 1
LDDMM_GRAD_JACOBI, LDDMM_GRAD_DISCRETE = 0, 1
LDDMM_TRACE_MAX = 64

STATUS = {
    0: "LDDMM_OK", 1: "LDDMM_ERR_ARG", 2: "LDDMM_ERR_SHAPE", 3: "LDDMM_ERR_OOM",
    4: "LDDMM_ERR_CUDA", 5: "LDDMM_ERR_NOT_LINEARIZED", 6: "LDDMM_ERR_NONFINITE",
    7: "LDDMM_ERR_DEVICE_CHECK", 8: "LDDMM_ERR_TIMEOUT", 9: "LDDMM_WARN_LINESEARCH",
    10: "LDDMM_ERR_TOO_LARGE",
}
LDDMM_WARN_LINESEARCH = 9


class lddmm_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("len", ctypes.c_double * 3)]


class lddmm_params(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("s", ctypes.c_int), ("weight", ctypes.c_double),
        ("nt", ctypes.c_int), ("interp", ctypes.c_int), ("space", ctypes.c_int),
        ("compute_dtype", ctypes.c_int), ("state_dtype", ctypes.c_int),
        ("checkpoint_every", ctypes.c_int), ("gn_maxit", ctypes.c_int), ("pcg_maxit", ctypes.c_int),
        ("pcg_rtol", ctypes.c_double), ("armijo_c1", ctypes.c_double), ("ls_maxit", ctypes.c_int),
        ("dealias", ctypes.c_int), ("optimizer", ctypes.c_int), ("gradient_mode", ctypes.c_int),
    ]


class lddmm_report(ctypes.Structure):
    _fields_ = [
        ("gn_iters", ctypes.c_int), ("pcg_iters_total", ctypes.c_int),
        ("mse_rel", ctypes.c_double), ("gnorm_rel", ctypes.c_double),
        ("jac_min", ctypes.c_double), ("jac_max", ctypes.c_double),
        ("energy", ctypes.c_double * (LDDMM_TRACE_MAX + 1)),
        ("pcg_iters", ctypes.c_int * LDDMM_TRACE_MAX),
        ("step", ctypes.c_double * LDDMM_TRACE_MAX),
    ]


class LddmmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = STATUS.get(status, str(status))
        try:
            msg += ": " + lib().lddmm_status_string(status).decode()
        except Exception:  # pragma: no cover - library not loadable
            pass
        super().__init__(f"{what}: {msg}" if what else msg)


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "lddmm_default_params": (None, [ctypes.POINTER(lddmm_params)]),
    "lddmm_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(lddmm_grid), ctypes.POINTER(lddmm_params)]),
    "lddmm_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(lddmm_grid), ctypes.POINTER(lddmm_params), _P]),
    "lddmm_destroy": (ctypes.c_int, [_P]),
    "lddmm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lddmm_last_status": (ctypes.c_int, [_P]),
    "lddmm_synchronize": (ctypes.c_int, [_P]),
    "lddmm_shoot": (ctypes.c_int, [_P, _P, _P, _P, _P, _D]),
    "lddmm_gradient": (ctypes.c_int, [_P, _P, _P, _P, _P, _D]),
    "lddmm_hessvec": (ctypes.c_int, [_P, _P, _P]),
    "lddmm_shoot_vjp": (ctypes.c_int, [_P, _P, _P]),
    "lddmm_jacobi_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "lddmm_jacobi_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "lddmm_apply_metric": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "lddmm_jacobian_det": (ctypes.c_int, [_P, _P, _P, _D]),
    "lddmm_register": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(lddmm_report)]),
    "lddmm_profile_num_classes": (ctypes.c_int, []),
    "lddmm_profile_class_name": (ctypes.c_char_p, [ctypes.c_int]),
    "lddmm_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "lddmm_profile_read": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, ctypes.POINTER(ctypes.c_longlong)]),
    "lddmm_apply_metric_noalloc": (ctypes.c_int, [ctypes.POINTER(lddmm_grid), ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "lddmm_apply_metric_noalloc_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(lddmm_grid), ctypes.c_int]),
    "lddmm_apply_metric_noalloc_capacity": (ctypes.c_size_t, []),
    "lddmm_probe_fp64_fma": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "lddmm_probe_fp64_fma_flops": (ctypes.c_double, [ctypes.c_int, ctypes.c_int]),
    "lddmm_probe_fp64_fma_threads": (ctypes.c_int, []),
}


def lib():
    """Load liblddmm.so (built in-tree by ``paper_1807_04638_gb300.build``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"liblddmm.so not found at {LIB_PATH}; build it with "
                "`python -m paper_1807_04638_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def default_params(**kw) -> lddmm_params:
    p = lddmm_params()
    lib().lddmm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def make_grid(n: Sequence[int], lengths: Optional[Sequence[float]] = None) -> lddmm_grid:
    g = lddmm_grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.len[a] = float(lengths[a]) if lengths is not None else 0.0
    return g


def workspace_bytes(n, params: lddmm_params, lengths=None) -> int:
    g = make_grid(n, lengths)
    return int(lib().lddmm_workspace_bytes(ctypes.byref(g), ctypes.byref(params)))


def _check(st: int, what: str, allow=()):
    if st != 0 and st not in allow:
        raise LddmmError(st, what)
    return st


def apply_metric_noalloc(x, out, power, alpha, s=2, lengths=None, stream=None):
    """out = L^power x through lddmm_apply_metric_noalloc (no device allocation).

    x, out: contiguous CUDA tensors [ncomp, n0, n1, n2] (or [n0, n1, n2]) of
    float64 or float32.  Raises LddmmError (LDDMM_ERR_TOO_LARGE) for grids
    whose scratch exceeds the library's fixed array.
    """
    import torch
    if x.dtype not in (torch.float64, torch.float32) or out.dtype != x.dtype:
        raise TypeError("x and out must both be float64 or both float32")
    if not (x.is_cuda and out.is_cuda and x.is_contiguous() and out.is_contiguous()) or x.shape != out.shape:
        raise ValueError("x and out must be contiguous CUDA tensors of the same shape")
    n = tuple(x.shape[-3:])
    ncomp = x.numel() // math.prod(n)
    g = make_grid(n, lengths)
    st = stream if stream is not None else torch.cuda.current_stream(x.device)
    dtype = LDDMM_F64 if x.dtype == torch.float64 else LDDMM_F32
    with torch.cuda.device(x.device):
        _check(lib().lddmm_apply_metric_noalloc(ctypes.byref(g), float(alpha), int(s), int(power), dtype,
                                                _P(x.data_ptr()), _P(out.data_ptr()), ncomp,
                                                _P(st.cuda_stream)), "lddmm_apply_metric_noalloc")


def probe_fp64_fma(device=None, blocks=None, iters=4096, reps=5) -> float:
    """Measured FP64 FMA rate in TFLOP/s (lddmm_probe_fp64_fma, CUDA events,
    best of `reps` launches after one warm-up)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    if blocks is None:
        blocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    thr = lib().lddmm_probe_fp64_fma_threads()
    out = torch.empty(blocks * thr, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    best = None
    with torch.cuda.device(dev):
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _check(lib().lddmm_probe_fp64_fma(_P(out.data_ptr()), blocks, iters, _P(st.cuda_stream)),
                   "lddmm_probe_fp64_fma")
            e1.record(st)
            torch.cuda.synchronize(dev)
            if r > 0:
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
    if not torch.isfinite(out).all():
        raise LddmmError(6, "lddmm_probe_fp64_fma")
    return lib().lddmm_probe_fp64_fma_flops(blocks, iters) / (best * 1e-3) / 1e12


class Handle:
    """One registration problem bound to a CUDA device and stream.

    Array arguments are torch CUDA tensors, contiguous, of the handle's
    compute dtype (float64 or float32), shaped [3, n0, n1, n2] (vector
    fields) or [n0, n1, n2] (images).  They are passed as raw device
    pointers; outputs are written in place.
    """

    def __init__(self, n, params: lddmm_params, lengths=None, stream=None, device=None):
        import torch
        self.torch = torch
        self.n = tuple(int(x) for x in n)
        self.params = params
        self.dtype = torch.float64 if params.compute_dtype == LDDMM_F64 else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._grid = make_grid(self.n, lengths)
            h = _P()
            _check(lib().lddmm_create(ctypes.byref(h), ctypes.byref(self._grid), ctypes.byref(params),
                                      _P(self.stream.cuda_stream)), "lddmm_create")
        self._h = h

    # -- marshalling helpers -------------------------------------------------
    def _ptr(self, t, shape, name, allow_none=False):
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        if not t.is_cuda or t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}, got {tuple(t.shape)}")
        return _P(t.data_ptr())

    def vec_shape(self):
        return (3,) + self.n

    def new_vec(self):
        return self.torch.empty(self.vec_shape(), dtype=self.dtype, device=self.device)

    def new_img(self):
        return self.torch.empty(self.n, dtype=self.dtype, device=self.device)

    # -- ABI calls -------------------------------------------------------------
    def lddmm_shoot(self, v0, I0=None, m1=None, u1=None, kinetic=False):
        kin = (ctypes.c_double * (self.params.nt + 1))() if kinetic else None
        _check(lib().lddmm_shoot(self._h, self._ptr(v0, self.vec_shape(), "v0"),
                                 self._ptr(I0, self.n, "I0", True), self._ptr(m1, self.n, "m1", True),
                                 self._ptr(u1, self.vec_shape(), "u1", True),
                                 ctypes.cast(kin, _D) if kin is not None else None), "lddmm_shoot")
        return list(kin) if kin is not None else None

    def lddmm_gradient(self, v0, I0, I1, grad, energy=True):
        e = (ctypes.c_double * 3)() if energy else None
        _check(lib().lddmm_gradient(self._h, self._ptr(v0, self.vec_shape(), "v0"), self._ptr(I0, self.n, "I0"),
                                    self._ptr(I1, self.n, "I1"), self._ptr(grad, self.vec_shape(), "grad"),
                                    ctypes.cast(e, _D) if e is not None else None), "lddmm_gradient")
        return tuple(e) if e is not None else None

    def lddmm_hessvec(self, dv0, Hdv):
        _check(lib().lddmm_hessvec(self._h, self._ptr(dv0, self.vec_shape(), "dv0"),
                                   self._ptr(Hdv, self.vec_shape(), "Hdv")), "lddmm_hessvec")

    def lddmm_shoot_vjp(self, G, out):
        _check(lib().lddmm_shoot_vjp(self._h, self._ptr(G, self.n, "G"), self._ptr(out, self.vec_shape(), "out")),
               "lddmm_shoot_vjp")

    def lddmm_jacobi_forward(self, dv0, eta1=None, xi1=None):
        _check(lib().lddmm_jacobi_forward(self._h, self._ptr(dv0, self.vec_shape(), "dv0"),
                                          self._ptr(eta1, self.vec_shape(), "eta1", True),
                                          self._ptr(xi1, self.vec_shape(), "xi1", True)), "lddmm_jacobi_forward")

    def lddmm_jacobi_adjoint(self, b_eta, b_xi, out):
        _check(lib().lddmm_jacobi_adjoint(self._h, self._ptr(b_eta, self.vec_shape(), "b_eta", True),
                                          self._ptr(b_xi, self.vec_shape(), "b_xi"),
                                          self._ptr(out, self.vec_shape(), "out")), "lddmm_jacobi_adjoint")

    def lddmm_apply_metric(self, x, out, power):
        ncomp = x.numel() // math.prod(self.n)
        shape = (ncomp,) + self.n if x.dim() == 4 else self.n
        _check(lib().lddmm_apply_metric(self._h, self._ptr(x, shape, "in"), self._ptr(out, shape, "out"),
                                        ncomp, int(power)), "lddmm_apply_metric")

    def lddmm_jacobian_det(self, u, J=None, minmax=True):
        mm = (ctypes.c_double * 2)() if minmax else None
        _check(lib().lddmm_jacobian_det(self._h, self._ptr(u, self.vec_shape(), "u"),
                                        self._ptr(J, self.n, "J", True),
                                        ctypes.cast(mm, _D) if mm is not None else None), "lddmm_jacobian_det")
        return tuple(mm) if mm is not None else None

    def lddmm_register(self, I0, I1, v0_inout):
        rep = lddmm_report()
        st = _check(lib().lddmm_register(self._h, self._ptr(I0, self.n, "I0"), self._ptr(I1, self.n, "I1"),
                                         self._ptr(v0_inout, self.vec_shape(), "v0_inout"), ctypes.byref(rep)),
                    "lddmm_register", allow=(LDDMM_WARN_LINESEARCH,))
        k = rep.gn_iters
        return {
            "status": STATUS[st], "gn_iters": k, "pcg_iters_total": rep.pcg_iters_total,
            "mse_rel": rep.mse_rel, "gnorm_rel": rep.gnorm_rel, "jac_min": rep.jac_min, "jac_max": rep.jac_max,
            "energy": list(rep.energy[:k + 1]), "pcg_iters": list(rep.pcg_iters[:k]), "step": list(rep.step[:k]),
        }

    def lddmm_profile(self, enable: bool):
        _check(lib().lddmm_profile(self._h, 1 if enable else 0), "lddmm_profile")

    def lddmm_profile_read(self):
        """{kernel class: (device ms, algorithmic bytes, launches)} since enable."""
        out = {}
        L = lib()
        for c in range(L.lddmm_profile_num_classes()):
            ms, by, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
            _check(L.lddmm_profile_read(self._h, c, ctypes.byref(ms), ctypes.byref(by), ctypes.byref(n)),
                   "lddmm_profile_read")
            out[L.lddmm_profile_class_name(c).decode()] = (ms.value, by.value, n.value)
        return out

    def lddmm_synchronize(self):
        _check(lib().lddmm_synchronize(self._h), "lddmm_synchronize")

    def close(self):
        if getattr(self, "_h", None):
            lib().lddmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
