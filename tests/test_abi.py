"""The C-ABI library loads without a GPU and exports every symbol the header
declares; host-side argument checks work without touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lddmm.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_1807_04638_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lddmm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lddmm_shoot", "lddmm_gradient", "lddmm_hessvec", "lddmm_register"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_checks_without_gpu(libpath):
    import paper_1807_04638_gb300 as pkg
    p = pkg.default_params()
    assert p.nt == 10 and p.s == 2 and abs(p.alpha - 0.01) < 1e-15
    b = pkg.workspace_bytes((32, 32, 32), p)
    assert b > 2 * 10 * 24 * 32 ** 3 * 8  # at least the stored time states
    p32 = pkg.default_params(compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    assert 0 < pkg.workspace_bytes((32, 32, 32), p32) < b
    # unsupported shapes and bad parameters are rejected before any device work
    assert pkg.workspace_bytes((7, 32, 32), p) == 0
    assert pkg.workspace_bytes((32, 32, 1024), p) == 0
    bad = pkg.default_params(nt=0)
    assert pkg.workspace_bytes((32, 32, 32), bad) == 0
    lib = pkg.lib()
    h = ctypes.c_void_p()
    g = pkg.make_grid((7, 8, 8))
    assert lib.lddmm_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(p), None) == 2  # SHAPE
    assert lib.lddmm_create(None, ctypes.byref(g), ctypes.byref(p), None) == 1  # ARG
    assert lib.lddmm_shoot(None, None, None, None, None, None) == 1
    assert lib.lddmm_status_string(5).decode().startswith("no linearisation")
    # parameter combinations the library refuses before any device work
    ok = pkg.default_params(compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    assert pkg.workspace_bytes((32, 32, 32), ok) > 0
    for kw in (dict(optimizer=2), dict(gradient_mode=2), dict(dealias=2), dict(checkpoint_every=0),
               dict(state_dtype=pkg.LDDMM_BF16, gradient_mode=pkg.LDDMM_GRAD_DISCRETE),
               dict(checkpoint_every=2, gradient_mode=pkg.LDDMM_GRAD_DISCRETE)):
        bad = pkg.default_params(compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
        for k, v in kw.items():
            setattr(bad, k, v)
        assert pkg.workspace_bytes((32, 32, 32), bad) == 0, kw
    # the exact discrete gradient keeps every map and every dE/dv_k
    ex = pkg.default_params(compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32,
                            gradient_mode=pkg.LDDMM_GRAD_DISCRETE)
    extra = pkg.workspace_bytes((32, 32, 32), ex) - pkg.workspace_bytes((32, 32, 32), ok)
    assert extra == (6 * (ok.nt + 1) + 6) * 32 ** 3 * 4
    # the FP64 rate probe checks its arguments before launching
    assert lib.lddmm_probe_fp64_fma(None, 1, 1, None) == 1
    thr = lib.lddmm_probe_fp64_fma_threads()
    assert lib.lddmm_probe_fp64_fma_flops(3, 5) == 2 * 8 * 5 * thr * 3


def test_autograd_memory_plan_without_gpu(libpath):
    """The differentiation form keeps every forward state while the batch's
    workspaces fit, else checkpoints every 2 steps (less than half the
    memory at nt = 10), else refuses."""
    import paper_1807_04638_gb300 as pkg
    from paper_1807_04638_gb300.autograd import Shooter
    p = pkg.default_params(compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32, nt=10)
    n = (96, 96, 96)
    full = pkg.workspace_bytes(n, p)
    assert Shooter.plan_memory(n, 8, p, 8 * full).checkpoint_every == 1
    q = Shooter.plan_memory(n, 8, p, 8 * full - 1)
    assert q.checkpoint_every == 2 and pkg.workspace_bytes(n, q) < 0.5 * full
    assert p.checkpoint_every == 1  # the caller's parameters are not changed
    with pytest.raises(MemoryError):
        Shooter.plan_memory(n, 8, p, 8 * pkg.workspace_bytes(n, q) - 1)
