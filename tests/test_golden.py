"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py
from the FP64 oracle alone).

* CPU: the oracle still reproduces the stored energy and gradient norm of
  the 32^3 plain-method workload at v0 = 0 (regression of the oracle);
* GPU: the FP64 library runs the whole plain-method registration of that
  workload (nt = 10, 5 Gauss-Newton x <= 10 PCG) with the oracle's
  decisions, energies and final metrics.
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


def _inputs():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg.config1_inputs()


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
