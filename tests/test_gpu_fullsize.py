"""GPU parity at the sizes the benchmark runs (register-blocked FFT passes).

* the metric operator and one gradient / Hessian product on 64^3 and mixed
  power-of-two grids, element by element against the FP64 oracle;
* the 128^3 workload in the benchmark's configuration (FP32 form, nt = 10,
  alpha = 0.005): the shooting outputs against the oracle, and for the
  Jacobi sweeps and the Gauss-Newton Hessian the properties that hold at any
  size (exact transposition, symmetry), since one oracle Hv at 128^3 takes
  minutes.
"""
import numpy as np
import pytest

from oracle import lddmm_oracle as O
from paper_1807_04638_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_04638_gb300 as p
    p.lib()
    return p


DT = {"f64": (torch.float64, 0), "f32": (torch.float32, 1)}


def dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [(128, 128, 128), (64, 256, 32), (256, 32, 64)])
def test_metric_large(pkg, prec, n):
    dtype, cd = DT[prec]
    g = O.Grid(n, alpha=0.005)
    f = synth.rng_for(21).standard_normal((3,) + n)
    tol = 1e-10 if prec == "f64" else 1e-5
    with pkg.Handle(n, pkg.default_params(alpha=0.005, compute_dtype=cd, state_dtype=cd)) as h:
        x = dev(f, dtype)
        out = torch.empty_like(x)
        h.lddmm_apply_metric(x, out, -1)
        h.lddmm_synchronize()
        assert rel(host(out), g.K(f)) < tol
        h.lddmm_apply_metric(x, out, 2)
        h.lddmm_synchronize()
        assert rel(host(out), g.L(g.L(f))) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gradient_hessvec_64(pkg, prec):
    dtype, cd = DT[prec]
    n = (64, 64, 64)
    nt = 3
    g = O.Grid(n, alpha=0.005)
    I0, vtrue = synth.blob_pair_inputs(n, 31, kmax=3, max_disp_vox=2.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, nt, I0).m1
    p = O.Params(alpha=0.005, nt=nt)
    v0 = 0.6 * vtrue
    gl2, E, _, _, tr = O.gradient(g, p, v0, I0, I1)
    d = synth.band_limited_field(n, synth.rng_for(32), 6.0, 3) * g.h[0]
    hl2 = O.hessvec(g, p, tr, d)
    tol = 1e-10 if prec == "f64" else 1e-5
    with pkg.Handle(n, pkg.default_params(alpha=0.005, nt=nt, compute_dtype=cd, state_dtype=cd)) as h:
        grad, hv = h.new_vec(), h.new_vec()
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        h.lddmm_hessvec(dev(d, dtype), hv)
        h.lddmm_synchronize()
    assert abs(e[0] - E) < tol * abs(E)
    assert rel(host(grad), O.to_space(g, p, gl2)) < tol
    assert rel(host(hv), O.to_space(g, p, hl2)) < tol


@pytest.fixture(scope="module")
def workload128():
    """The 128^3 benchmark workload (same recipe and seeds as bench.py)."""
    import bench
    return bench.workload_inputs()


def test_shoot_128_bench_configuration(pkg, workload128):
    P, v0t, e0, e1, d = workload128
    n = (128, 128, 128)
    g = O.Grid(n, alpha=0.005)
    v0 = 0.5 * v0t
    tr = O.shoot(g, v0, 10, P)
    prm = pkg.default_params(alpha=0.005, nt=10, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    with pkg.Handle(n, prm) as h:
        m1, u1 = h.new_img(), h.new_vec()
        kin = h.lddmm_shoot(dev(v0, torch.float32), dev(P, torch.float32), m1, u1, kinetic=True)
    assert rel(host(u1), tr.u) < 1e-5
    assert rel(host(m1) - P, tr.m1 - P) < 1e-4
    assert np.allclose(kin, tr.kinetic, rtol=1e-5, atol=0)


def test_sweeps_and_hessian_properties_128(pkg, workload128):
    P, v0t, e0, e1, d = workload128
    n = (128, 128, 128)
    r = synth.rng_for(40)
    prm = pkg.default_params(alpha=0.005, nt=10, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32,
                             space=pkg.LDDMM_SPACE_L2)
    f32 = torch.float32
    with pkg.Handle(n, prm) as h:
        I0 = dev(P + e0, f32)
        I1 = dev(np.roll(P, 3, axis=0) + e1, f32)
        grad = h.new_vec()
        e = h.lddmm_gradient(dev(0.5 * v0t, f32), I0, I1, grad)
        assert np.isfinite(e).all()
        x = dev(synth.band_limited_field(n, r, 20.0, 3), f32)
        y = dev(synth.band_limited_field(n, r, 20.0, 3), f32)
        be = dev(r.standard_normal((3,) + n), f32)
        bx = dev(r.standard_normal((3,) + n), f32)
        e1_, x1_, a0 = h.new_vec(), h.new_vec(), h.new_vec()
        h.lddmm_jacobi_forward(x, e1_, x1_)
        h.lddmm_jacobi_adjoint(be, bx, a0)
        hx, hy = h.new_vec(), h.new_vec()
        h.lddmm_hessvec(x, hx)
        h.lddmm_hessvec(y, hy)
        h.lddmm_synchronize()
    X, Y = host(x), host(y)
    lhs = np.sum(host(e1_) * host(be)) + np.sum(host(x1_) * host(bx))
    rhs = np.sum(X * host(a0))
    assert abs(lhs - rhs) < 1e-5 * (abs(lhs) + abs(rhs))
    hxy, xhy = np.sum(host(hx) * Y), np.sum(X * host(hy))
    assert abs(hxy - xhy) < 1e-5 * (abs(hxy) + abs(xhy))
    assert np.sum(host(hx) * X) > 0 and np.isfinite(host(hx)).all()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [(96, 40, 32), (40, 96, 160), (192, 36, 48)])
def test_mixed_radix_compiled_sizes(pkg, prec, n):
    """Gradient and Hv on grids whose axes use the compiled 96/160/192 plans."""
    dtype, cd = DT[prec]
    nt = 2
    g = O.Grid(n, alpha=0.01)
    I0, vtrue = synth.blob_pair_inputs(n, 41, kmax=3, max_disp_vox=1.5)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, nt, I0).m1
    p = O.Params(nt=nt)
    v0 = 0.5 * vtrue
    gl2, E, _, _, tr = O.gradient(g, p, v0, I0, I1)
    d = synth.band_limited_field(n, synth.rng_for(42), 6.0, 3) * g.h[0]
    hl2 = O.hessvec(g, p, tr, d)
    tol = 1e-10 if prec == "f64" else 1e-5
    with pkg.Handle(n, pkg.default_params(nt=nt, compute_dtype=cd, state_dtype=cd)) as h:
        grad, hv = h.new_vec(), h.new_vec()
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        h.lddmm_hessvec(dev(d, dtype), hv)
        h.lddmm_synchronize()
    assert abs(e[0] - E) < tol * abs(E)
    assert rel(host(grad), O.to_space(g, p, gl2)) < tol
    assert rel(host(hv), O.to_space(g, p, hl2)) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_metric_160_192_96(pkg, prec):
    dtype, cd = DT[prec]
    n = (160, 192, 96)
    g = O.Grid(n, alpha=0.005)
    f = synth.rng_for(43).standard_normal((3,) + n)
    tol = 1e-10 if prec == "f64" else 1e-5
    with pkg.Handle(n, pkg.default_params(alpha=0.005, compute_dtype=cd, state_dtype=cd)) as h:
        x = dev(f, dtype)
        out = torch.empty_like(x)
        h.lddmm_apply_metric(x, out, -1)
        h.lddmm_synchronize()
        assert rel(host(out), g.K(f)) < tol


def test_band_limited_passes_equal_full_transforms(pkg, workload128, monkeypatch):
    """With the 2/3-rule projector the shooting and Jacobi-sweep transforms
    touch only the band; the results equal those of full transforms (the
    skipped entries are zero or only ever used through P).  Both runs use
    the separate axis-2 passes (the full transforms have no fused stage);
    the fused stages are compared with them in test_gpu_fused.py."""
    P, v0t, e0, e1, d = workload128
    n = (128, 128, 128)
    f32 = torch.float32
    prm = pkg.default_params(alpha=0.005, nt=10, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    out = {}
    monkeypatch.setenv("LDDMM_UNFUSED", "1")
    for mode in ("band", "full"):
        if mode == "full":
            monkeypatch.setenv("LDDMM_FULL_BAND", "1")
        else:
            monkeypatch.delenv("LDDMM_FULL_BAND", raising=False)
        monkeypatch.setenv("LDDMM_POISON_WORKSPACE", "1")
        with pkg.Handle(n, prm) as h:
            grad, hv, xi1, a0 = h.new_vec(), h.new_vec(), h.new_vec(), h.new_vec()
            e = h.lddmm_gradient(dev(0.5 * v0t, f32), dev(P + e0, f32), dev(P + e1, f32), grad)
            h.lddmm_hessvec(dev(d, f32), hv)
            h.lddmm_jacobi_forward(dev(d, f32), None, xi1)
            h.lddmm_jacobi_adjoint(None, dev(d, f32), a0)
            h.lddmm_synchronize()
            out[mode] = (e, host(grad), host(hv), host(xi1), host(a0))
    eb, ef = out["band"][0], out["full"][0]
    assert np.allclose(eb, ef, rtol=1e-12, atol=0)
    for a, b in zip(out["band"][1:], out["full"][1:]):
        assert np.isfinite(a).all()
        assert rel(a, b) < 1e-6, rel(a, b)


_BAND_CASES = {}


def _band_case(n):
    """Oracle results for the band-limited grid tests (computed once per grid)."""
    if n not in _BAND_CASES:
        nt = 3
        g = O.Grid(n, alpha=0.01)
        I0, vtrue = synth.blob_pair_inputs(n, 51, kmax=3, max_disp_vox=1.5)
        I0 = synth.spectral_gaussian_smooth(I0, 1.0)
        I1 = O.shoot(g, vtrue, nt, I0).m1
        p = O.Params(nt=nt)
        v0 = 0.5 * vtrue
        gl2, E, _, _, tr = O.gradient(g, p, v0, I0, I1)
        r = synth.rng_for(52)
        dvec = synth.band_limited_field(n, r, 6.0, 3) * g.h[0]
        be, bx = r.standard_normal((3,) + n), r.standard_normal((3,) + n)
        want = dict(E=E, grad=O.to_space(g, p, gl2), hv=O.to_space(g, p, O.hessvec(g, p, tr, dvec)),
                    tan=O.tangent(g, tr, dvec), adj=O.adjoint(g, tr, bx, be))
        _BAND_CASES[n] = (nt, I0, I1, v0, dvec, be, bx, want)
    return _BAND_CASES[n]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [(32, 64, 96), (96, 32, 64)])
def test_band_limited_grids_vs_oracle(pkg, prec, n, monkeypatch):
    """Grids whose three axes all use compiled plans (band-limited passes),
    with a NaN-poisoned workspace: gradient, Hv and both sweeps against the
    oracle."""
    monkeypatch.setenv("LDDMM_POISON_WORKSPACE", "1")
    monkeypatch.delenv("LDDMM_FULL_BAND", raising=False)
    dtype, cd = DT[prec]
    nt, I0, I1, v0, dvec, be, bx, want = _band_case(n)
    tol = 1e-10 if prec == "f64" else 1e-5
    with pkg.Handle(n, pkg.default_params(nt=nt, compute_dtype=cd, state_dtype=cd)) as h:
        grad, hv, e1g, x1g, a0g = (h.new_vec() for _ in range(5))
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        h.lddmm_hessvec(dev(dvec, dtype), hv)
        h.lddmm_jacobi_forward(dev(dvec, dtype), e1g, x1g)
        h.lddmm_jacobi_adjoint(dev(be, dtype), dev(bx, dtype), a0g)
        h.lddmm_synchronize()
    assert abs(e[0] - want["E"]) < tol * abs(want["E"])
    assert rel(host(grad), want["grad"]) < tol
    assert rel(host(hv), want["hv"]) < tol
    assert rel(host(e1g), want["tan"][0]) < tol
    assert rel(host(x1g), want["tan"][1]) < tol
    assert rel(host(a0g), want["adj"]) < tol


def test_brain_shaped_grid_metric_full_array_and_shoot_vs_oracle(pkg):
    """The 256x300x256 grid of the brain-shaped workload: its n1 = 300 axis
    (2^2 3 5^2) runs the runtime-radix passes.  K and L on a field against
    the oracle over the whole array (FP32 1e-5, FP64 1e-10); the FP32 shoot
    (nt = 2, FP32 states) against the oracle's stored samples, complete
    planes, norms and kinetic energies (tests/golden/make_golden.py config3);
    the precision form's shoot (bfloat16 states, checkpointed) reported
    against the same values at its own tolerance (reading C14)."""
    import importlib.util
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    n, nt, alpha = mg.C3_N, mg.C3_NT, mg.C3_ALPHA
    g = O.Grid(n, alpha=alpha)
    f = synth.band_limited_field(n, synth.rng_for(301), 10.0, 3) + 0.05 * synth.rng_for(302).standard_normal((3,) + n)
    for prec, tol in (("f64", 1e-10), ("f32", 1e-5)):
        dtype, cd = DT[prec]
        with pkg.Handle(n, pkg.default_params(alpha=alpha, nt=1, compute_dtype=cd, state_dtype=cd)) as h:
            x = dev(f, dtype)
            out = torch.empty_like(x)
            h.lddmm_apply_metric(x, out, -1)
            h.lddmm_synchronize()
            assert rel(host(out), g.K(f)) < tol, prec
            h.lddmm_apply_metric(x, out, 1)
            h.lddmm_synchronize()
            assert rel(host(out), g.L(f)) < tol, prec
            del x, out
    with open(os.path.join(here, "golden", "config3_256x300x256.json")) as fh:
        ref = json.load(fh)
    planes = np.load(os.path.join(here, "golden", "config3_planes.npz"))
    I0, v0t = mg.config3_inputs()
    idx = mg.config3_sample_idx()
    assert [int(i) for i in idx] == ref["idx"]
    f32 = torch.float32
    for states, ckpt, tol in ((pkg.LDDMM_F32, 1, 1e-5), (pkg.LDDMM_BF16, 2, 2e-2)):
        prm = pkg.default_params(alpha=alpha, nt=nt, compute_dtype=pkg.LDDMM_F32, state_dtype=states,
                                 checkpoint_every=ckpt)
        with pkg.Handle(n, prm) as h:
            m1, u1 = h.new_img(), h.new_vec()
            kin = h.lddmm_shoot(dev(v0t, f32), dev(I0, f32), m1, u1, kinetic=True)
            h.lddmm_synchronize()
            un, mn = host(u1), host(m1)
        assert rel(un.ravel()[idx], ref["u1"]) < tol, (states, rel(un.ravel()[idx], ref["u1"]))
        assert rel(mn.ravel()[idx % mn.size], ref["m1"]) < tol
        assert abs(np.linalg.norm(un) - ref["u1_l2"]) < tol * ref["u1_l2"]
        assert abs(np.linalg.norm(mn) - ref["m1_l2"]) < tol * ref["m1_l2"]
        assert np.allclose(kin, ref["kinetic"], rtol=tol, atol=0)
        if states == pkg.LDDMM_F32:
            for axis, i in mg.C3_U_PLANES:
                assert rel(np.take(un, i, axis=1 + axis), planes[f"u1_axis{axis}_{i}"]) < tol, (axis, i)
            for axis, i in mg.C3_M_PLANES:
                assert rel(np.take(mn, i, axis=axis), planes[f"m1_axis{axis}_{i}"]) < tol, (axis, i)
