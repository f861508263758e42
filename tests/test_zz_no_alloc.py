"""The no-allocation metric entry point agrees with the handle's metric apply
and with the FP64 oracle.

lddmm_apply_metric_noalloc serves callers that cannot allocate device memory
(graph capture, real-time loops, plug-ins whose host owns all allocations):
its scratch is a fixed array inside the library.  Two calls in a row must both
match lddmm_apply_metric of a handle (which uses its own allocated
workspace), within the parity tolerances of the suite, so a second call is
not affected by what the first left in the shared scratch.  This file is
collected last and must also pass when run alone in a fresh process, where
its first call performs the per-device set-up.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_04638_gb300 as p
    p.lib()
    return p


def rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-5)])
def test_noalloc_matches_handle_two_calls_in_a_row(pkg, dtype, tol):
    n = (64, 48, 40)           # power-of-two and mixed-radix axes
    alpha, s = 0.005, 2
    g = torch.Generator(device="cpu").manual_seed(7)
    xa = torch.randn((3,) + n, generator=g, dtype=torch.float64).to("cuda", dtype)
    xb = torch.randn((3,) + n, generator=g, dtype=torch.float64).to("cuda", dtype)
    cd = pkg.LDDMM_F64 if dtype == torch.float64 else pkg.LDDMM_F32
    with pkg.Handle(n, pkg.default_params(alpha=alpha, s=s, compute_dtype=cd, state_dtype=cd)) as h:
        ref_a, ref_b = torch.empty_like(xa), torch.empty_like(xb)
        h.lddmm_apply_metric(xa, ref_a, -1)
        h.lddmm_apply_metric(xb, ref_b, 2)
        h.lddmm_synchronize()
    out_a, out_b = torch.empty_like(xa), torch.empty_like(xb)
    pkg.apply_metric_noalloc(xa, out_a, -1, alpha, s)
    pkg.apply_metric_noalloc(xb, out_b, 2, alpha, s)
    torch.cuda.synchronize()
    assert rel(out_a, ref_a) < tol
    assert rel(out_b, ref_b) < tol
    # and directly against the FP64 oracle: K = L^-1 and L^2
    from oracle import lddmm_oracle as O
    go = O.Grid(n, alpha=alpha, s=s)
    want_a = torch.from_numpy(go.K(xa.double().cpu().numpy()))
    want_b = torch.from_numpy(go.L(go.L(xb.double().cpu().numpy())))
    assert rel(out_a.double().cpu(), want_a) < tol
    assert rel(out_b.double().cpu(), want_b) < tol
    # in place (out == in) gives the same result
    xc = xa.clone()
    pkg.apply_metric_noalloc(xc, xc, -1, alpha, s)
    torch.cuda.synchronize()
    assert rel(xc, ref_a) < tol


def test_noalloc_rejects_grids_beyond_its_scratch(pkg):
    lib = pkg.lib()
    cap = lib.lddmm_apply_metric_noalloc_capacity()
    g128 = pkg.make_grid((128, 128, 128))
    assert lib.lddmm_apply_metric_noalloc_scratch_bytes(ctypes.byref(g128), pkg.LDDMM_F32) <= cap
    assert lib.lddmm_apply_metric_noalloc_scratch_bytes(ctypes.byref(g128), pkg.LDDMM_F64) > cap
    x = torch.zeros((128, 128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LddmmError) as ei:
        pkg.apply_metric_noalloc(x, x, -1, 0.005, 2)
    assert ei.value.status == 10  # LDDMM_ERR_TOO_LARGE
