"""The Hessian-vector product replays a recorded CUDA graph of its launches
when the handle's stream can be captured: its results equal those of the
launches issued one by one (LDDMM_NO_GRAPH=1) bit for bit, after a change of
the input and output buffers (a new recording), and inside a whole
registration (PCG calls it with fixed buffers).  On the legacy default
stream the launches run one by one with the same results."""
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


def run(pkg, n, prm, I0, I1, v0, dirs, use_default_stream=False):
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    st = torch.cuda.default_stream() if use_default_stream else torch.cuda.Stream()
    with torch.cuda.stream(st):
        with pkg.Handle(n, prm, stream=st) as h:
            g = h.new_vec()
            h.lddmm_gradient(T(v0), T(I0), T(I1), g)
            outs = []
            d0, o0 = T(dirs[0]), h.new_vec()
            for _ in range(3):  # same buffers: recorded once, replayed
                h.lddmm_hessvec(d0, o0)
            outs.append(o0.clone())
            d1, o1 = T(dirs[1]), h.new_vec()  # new buffers: recorded again
            h.lddmm_hessvec(d1, o1)
            outs.append(o1.clone())
            h.lddmm_hessvec(d0, o0)
            outs.append(o0.clone())
            v = torch.zeros((3,) + n, dtype=torch.float32, device="cuda")
            rep = h.lddmm_register(T(I0), T(I1), v)
            torch.cuda.synchronize()
    return outs, v, rep


@pytest.mark.parametrize("n", [(32, 32, 32), (64, 32, 128)])
def test_graph_replay_equals_launches_one_by_one(pkg, n, monkeypatch):
    I0, vt = synth.blob_pair_inputs(n, 41, kmax=3, max_disp_vox=2.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = np.roll(I0, 1, axis=2)
    dirs = [synth.band_limited_field(n, synth.rng_for(42 + i), 4.0, 3) * (2 * np.pi / n[0]) for i in range(2)]
    prm = pkg.default_params(alpha=0.01, nt=4, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32,
                             gn_maxit=2, pcg_maxit=5)
    monkeypatch.delenv("LDDMM_NO_GRAPH", raising=False)
    graph = run(pkg, n, prm, I0, I1, 0.5 * vt, dirs)
    legacy = run(pkg, n, prm, I0, I1, 0.5 * vt, dirs, use_default_stream=True)
    monkeypatch.setenv("LDDMM_NO_GRAPH", "1")
    plain = run(pkg, n, prm, I0, I1, 0.5 * vt, dirs)
    for other in (plain, legacy):
        for a, b in zip(graph[0], other[0]):
            assert torch.equal(a, b)
        assert torch.equal(graph[1], other[1])
        assert graph[2]["pcg_iters"] == other[2]["pcg_iters"] and graph[2]["energy"] == other[2]["energy"]
