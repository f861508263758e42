"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py
from the FP64 oracle alone).

* CPU: the oracle still reproduces the stored energy and gradient norm of
  the 32^3 plain-method workload at v0 = 0 (regression of the oracle);
* GPU: the FP64 library runs the whole plain-method registration of that
  workload (nt = 10, 5 Gauss-Newton x <= 10 PCG) with the oracle's
  decisions, energies and final metrics;
* GPU: on the 128^3 benchmark workload, in the configuration the benchmark
  times (FP32 form, nt = 10), the V gradient and the V Hessian-vector
  product match the oracle at 2048 stored sample points and on stored
  complete planes along each axis; the target rebuilt on the GPU in FP64 is
  checked against the oracle's stored samples first.
"""
import json
import os

import numpy as np
import pytest

from oracle import lddmm_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "config1_register_32cubed.json")


def _load():
    with open(GOLDEN) as f:
        return json.load(f)


def _mg():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def _inputs():
    return _mg().config1_inputs()


def test_oracle_reproduces_stored_config1_start():
    ref = _load()
    g, p, I0, I1 = _inputs()
    zero = np.zeros((3,) + g.n)
    g0, E0 = O.gradient(g, p, zero, I0, I1)[:2]
    assert abs(E0 - ref["E_at_zero"]) < 1e-12 * ref["E_at_zero"]
    assert abs(np.sqrt(g.dot(g0, g0)) - ref["grad_L2_norm_at_zero"]) < 1e-12 * ref["grad_L2_norm_at_zero"]


@pytest.mark.gpu
def test_gpu_config1_registration_matches_stored_trace():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_04638_gb300 as pkg
    ref = _load()
    g, p, I0, I1 = _inputs()
    prm = pkg.default_params(alpha=0.01, nt=10, weight=1e-3, gn_maxit=5, pcg_maxit=10, pcg_rtol=0.1)
    f64 = torch.float64
    with pkg.Handle(g.n, prm) as h:
        v = torch.zeros((3,) + g.n, dtype=f64, device="cuda")
        rep = h.lddmm_register(torch.tensor(I0, dtype=f64, device="cuda"),
                               torch.tensor(I1, dtype=f64, device="cuda"), v)
        vn = v.cpu().numpy()
    assert rep["pcg_iters"] == ref["pcg_iters"] and rep["step"] == ref["steps"]
    assert np.allclose(rep["energy"], ref["energies"], rtol=1e-9, atol=0)
    for k in ("mse_rel", "gnorm_rel", "jac_min", "jac_max"):
        assert abs(rep[k] - ref[k]) < 1e-9 * max(1.0, abs(ref[k])), k
    assert abs(np.sqrt(g.dot(vn, vn)) - ref["v0_l2_norm"]) < 1e-9 * ref["v0_l2_norm"]


@pytest.mark.gpu
def test_gpu_bench128_gradient_and_hv_at_sampled_points():
    """Full size, benchmark configuration: the FP32 V gradient and V Hv at
    v0 = v0_true / 2 against the oracle at the stored sample points (relative
    L2 over the samples 1e-5), and the energy and full-array norms to 1e-5."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_04638_gb300 as pkg
    with open(os.path.join(HERE, "golden", "bench128_samples.json")) as f:
        ref = json.load(f)
    n, P, v0t, e0, e1, d, idx = _mg().bench128_inputs()
    assert [int(i) for i in idx] == ref["idx"]
    f64, f32 = torch.float64, torch.float32
    # target: the FP64 library shoot of the true velocity (the oracle's to
    # about 1e-10) plus the stored-recipe noise
    with pkg.Handle(n, pkg.default_params(alpha=0.005, nt=10)) as h64:
        m1 = h64.new_img()
        h64.lddmm_shoot(torch.tensor(v0t, dtype=f64, device="cuda"), torch.tensor(P, dtype=f64, device="cuda"), m1)
        h64.lddmm_synchronize()
        m1t = m1.cpu().numpy()
    # the rebuilt target is the oracle's (stored samples and norm) to 1e-9
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))
    assert rel(m1t.ravel()[idx % m1t.size], ref["m1_true"]) < 1e-9
    assert abs(np.linalg.norm(m1t) - ref["m1_true_l2"]) < 1e-9 * ref["m1_true_l2"]
    I1 = m1t + e1
    prm = pkg.default_params(alpha=0.005, nt=10, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=f32, device="cuda")
    with pkg.Handle(n, prm) as h:
        grad, hv = h.new_vec(), h.new_vec()
        e = h.lddmm_gradient(T(0.5 * v0t), T(P + e0), T(I1), grad)
        h.lddmm_hessvec(T(d), hv)
        h.lddmm_synchronize()
        gn, hn = grad.double().cpu().numpy(), hv.double().cpu().numpy()
    assert abs(e[0] - ref["E"]) < 1e-5 * ref["E"]
    assert rel(gn.ravel()[idx], ref["grad_V"]) < 1e-5
    assert rel(hn.ravel()[idx], ref["hv_V"]) < 1e-5
    assert abs(np.linalg.norm(gn) - ref["grad_V_l2"]) < 1e-5 * ref["grad_V_l2"]
    assert abs(np.linalg.norm(hn) - ref["hv_V_l2"]) < 1e-5 * ref["hv_V_l2"]
    # complete planes across every tile of the other two axes
    planes = np.load(os.path.join(HERE, "golden", "bench128_planes.npz"))
    mg = _mg()
    for name, field, cuts in (("hv_V", hn, mg.BENCH128_HV_PLANES), ("grad_V", gn, mg.BENCH128_GRAD_PLANES)):
        for axis, i in cuts:
            want = planes[f"{name}_axis{axis}_{i}"]
            assert rel(np.take(field, i, axis=1 + axis), want) < 1e-5, (name, axis, i)
