"""Serving form: continuous batching with admission by HBM budget.

* every result is the same alone (serial run) and in the concurrent mix;
* admission respects the HBM budget (peak live workspace <= budget) while
  requests overlap;
* a request with non-finite data, and one that can never fit the budget,
  fail with an error status while the others complete unchanged.
"""
import numpy as np
import pytest

from paper_1807_04638_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_04638_gb300 as p
    p.lib()
    return p


def make_requests(pkg, specs):
    from paper_1807_04638_gb300.serve import Request
    reqs = []
    for i, (n, seed) in enumerate(specs):
        I0, vt = synth.blob_pair_inputs(n, seed, kmax=2, max_disp_vox=1.5)
        I0 = synth.spectral_gaussian_smooth(I0, 1.0)
        I1 = np.roll(synth.spectral_gaussian_smooth(I0, 1.5), 1, axis=0)
        prm = pkg.default_params(nt=4, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32,
                                 gn_maxit=3, pcg_maxit=8)
        reqs.append(Request(rid=i, I0=I0, I1=I1, params=prm, arrival=0.05 * i))
    return reqs


SPECS = [((32, 32, 32), 1), ((24, 32, 40), 2), ((48, 48, 48), 3), ((32, 32, 32), 4), ((40, 24, 32), 5)]


def test_alone_equals_mixed(pkg):
    from paper_1807_04638_gb300.serve import Server, serial, latency_stats
    reqs = make_requests(pkg, SPECS)
    alone = serial(reqs)
    srv = Server(budget_bytes=64e9, max_inflight=4)
    try:
        mixed = srv.run_trace(reqs)
    finally:
        srv.close()
    assert srv.peak_inflight > 1
    for a, m in zip(alone, mixed):
        assert a.status == "LDDMM_OK" and m.status == "LDDMM_OK", (a.status, m.status)
        err = np.linalg.norm(a.v0 - m.v0) / np.linalg.norm(a.v0)
        assert err <= 1e-6, (a.rid, err)
        assert a.report["pcg_iters"] == m.report["pcg_iters"]
    st = latency_stats(mixed)
    assert st["completed"] == len(reqs) and st["p99_s"] >= st["p50_s"] > 0


def test_admission_by_budget(pkg):
    from paper_1807_04638_gb300.serve import Server
    reqs = make_requests(pkg, SPECS)
    need = max(pkg.workspace_bytes(r.I0.shape, r.params) for r in reqs)
    budget = 1.5 * need  # room for one large or a couple of small handles
    srv = Server(budget_bytes=budget, max_inflight=8)
    try:
        res = srv.run_trace(reqs)
    finally:
        srv.close()
    assert all(r.status == "LDDMM_OK" for r in res), [(r.rid, r.status) for r in res]
    assert srv.peak_used <= budget


def test_faulty_requests_fail_alone(pkg):
    from paper_1807_04638_gb300.serve import Server, serial
    reqs = make_requests(pkg, SPECS[:3])
    good = serial(reqs)
    bad = make_requests(pkg, [((32, 32, 32), 9)])[0]
    bad.rid = 10
    bad.I0 = bad.I0.copy()
    bad.I0[3, 4, 5] = np.nan
    huge = make_requests(pkg, [((32, 32, 32), 9)])[0]
    huge.rid = 11
    srv = Server(budget_bytes=1.2 * pkg.workspace_bytes((48, 48, 48), reqs[0].params), max_inflight=4)
    huge.params = pkg.default_params(nt=40, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    huge.I0 = np.zeros((160, 192, 160))
    huge.I1 = np.zeros((160, 192, 160))
    try:
        res = srv.run_trace(reqs + [bad, huge])
    finally:
        srv.close()
    byid = {r.rid: r for r in res}
    assert byid[10].status.startswith("error")
    assert byid[11].status.startswith("error") and "budget" in byid[11].status
    for g in good:
        m = byid[g.rid]
        assert m.status == "LDDMM_OK"
        assert np.linalg.norm(g.v0 - m.v0) <= 1e-6 * np.linalg.norm(g.v0)
