"""GPU path vs the FP64 CPU oracle, through the C ABI, element by element.

Tolerances (relative L2 over the whole array, computed in FP64):
  FP64 engine: 1e-10 on every array output.
  FP32 engine: 1e-5 on gradients and Hessian products, 1e-4 on m(1) - I1 and
  on det(I + D u1).
Grids span several FFT tiles with ragged tails, radices 2, 3, 5 and an odd
last axis.
"""
import math

import numpy as np
import pytest

from oracle import lddmm_oracle as O
from paper_1807_04638_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-10


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


def dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


DT = {"f64": (torch.float64, 0), "f32": (torch.float32, 1)}


def params(pkg, prec, **kw):
    _, cd = DT[prec]
    return pkg.default_params(compute_dtype=cd, state_dtype=cd, **kw)


def problem(n, seed, nt, disp=1.0, kmax=2):
    g = O.Grid(n, alpha=0.01)
    I0, vtrue = synth.blob_pair_inputs(n, seed, kmax=kmax, max_disp_vox=disp)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, nt, I0).m1
    return g, I0, I1, vtrue


GRIDS = [(20, 12, 18), (12, 10, 15), (32, 32, 32)]


# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [(20, 12, 18), (12, 10, 15), (6, 4, 8)])
def test_apply_metric(pkg, prec, n):
    dtype, _ = DT[prec]
    g = O.Grid(n, alpha=0.03, lengths=(1.0, 2.0, 3.0))
    f = synth.rng_for(1).standard_normal((3,) + n)
    tol = F64_TOL if prec == "f64" else 1e-5
    with pkg.Handle(n, params(pkg, prec, alpha=0.03), lengths=(1.0, 2.0, 3.0)) as h:
        x = dev(f, dtype)
        out = torch.empty_like(x)
        for power, ref in ((-1, g.K(f)), (1, g.L(f)), (0, f)):
            h.lddmm_apply_metric(x, out, power)
            h.lddmm_synchronize()
            assert rel(host(out), ref) < tol, (power, rel(host(out), ref))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", GRIDS)
def test_shoot(pkg, prec, n):
    dtype, _ = DT[prec]
    nt = 6
    g, I0, I1, vtrue = problem(n, 3, nt)
    v0 = 0.8 * vtrue  # so that the residual m(1) - I1 is not zero
    tr = O.shoot(g, v0, nt, I0)
    with pkg.Handle(n, params(pkg, prec, nt=nt)) as h:
        m1 = h.new_img()
        u1 = h.new_vec()
        kin = h.lddmm_shoot(dev(v0, dtype), dev(I0, dtype), m1, u1, kinetic=True)
    tol_u = F64_TOL if prec == "f64" else 1e-5
    tol_m = F64_TOL if prec == "f64" else 1e-4
    assert rel(host(u1), tr.u) < tol_u
    assert rel(host(m1) - I1, tr.m1 - I1) < tol_m
    assert np.allclose(kin, tr.kinetic, rtol=F64_TOL if prec == "f64" else 1e-5, atol=0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("space", ["V", "L2"])
@pytest.mark.parametrize("n", GRIDS)
def test_gradient_and_hessvec(pkg, prec, space, n):
    dtype, _ = DT[prec]
    nt = 5
    g, I0, I1, vtrue = problem(n, 4, nt)
    p = O.Params(nt=nt, space=space)
    v0 = 0.5 * vtrue
    gl2, E, data, reg, tr = O.gradient(g, p, v0, I0, I1)
    d = synth.band_limited_field(n, synth.rng_for(7), 3.0, 3) * g.h[0]
    hl2 = O.hessvec(g, p, tr, d)
    sp = pkg.LDDMM_SPACE_V if space == "V" else pkg.LDDMM_SPACE_L2
    tol = F64_TOL if prec == "f64" else 1e-5
    with pkg.Handle(n, params(pkg, prec, nt=nt, space=sp)) as h:
        grad = h.new_vec()
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        hv = h.new_vec()
        h.lddmm_hessvec(dev(d, dtype), hv)
        h.lddmm_synchronize()
    assert abs(e[0] - E) < tol * abs(E) and abs(e[1] - data) < tol * abs(data) and abs(e[2] - reg) < tol * abs(reg)
    assert rel(host(grad), O.to_space(g, p, gl2)) < tol
    assert rel(host(hv), O.to_space(g, p, hl2)) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gradient_and_hessvec_rows_wider_than_a_block(pkg, prec):
    """Spectral rows of 288 entries along k1 (2^5 3^2, a runtime-radix axis),
    more than the 256 threads with which the spectral combination kernel
    walks a row, so that its threads take several entries of a row."""
    dtype, _ = DT[prec]
    n = (8, 288, 16)
    nt = 3
    g, I0, I1, vtrue = problem(n, 11, nt)
    p = O.Params(nt=nt)
    v0 = 0.5 * vtrue
    gl2, E, data, reg, tr = O.gradient(g, p, v0, I0, I1)
    d = synth.band_limited_field(n, synth.rng_for(12), 3.0, 3) * g.h[0]
    hl2 = O.hessvec(g, p, tr, d)
    tol = F64_TOL if prec == "f64" else 1e-5
    with pkg.Handle(n, params(pkg, prec, nt=nt)) as h:
        grad = h.new_vec()
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        hv = h.new_vec()
        h.lddmm_hessvec(dev(d, dtype), hv)
        h.lddmm_synchronize()
    assert abs(e[0] - E) < tol * abs(E)
    assert rel(host(grad), O.to_space(g, p, gl2)) < tol
    assert rel(host(hv), O.to_space(g, p, hl2)) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_jacobi_sweeps_and_dot_test(pkg, prec):
    dtype, _ = DT[prec]
    n = (20, 12, 18)
    nt = 4
    g, I0, I1, vtrue = problem(n, 5, nt)
    p = O.Params(nt=nt)
    v0 = 0.7 * vtrue
    tr = O.gradient(g, p, v0, I0, I1)[4]
    r = synth.rng_for(9)
    d, be, bx = (r.standard_normal((3,) + n) for _ in range(3))
    eta, xi = O.tangent(g, tr, d)
    adj = O.adjoint(g, tr, bx, be)
    tol = F64_TOL if prec == "f64" else 1e-5
    with pkg.Handle(n, params(pkg, prec, nt=nt)) as h:
        grad = h.new_vec()
        h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad, energy=False)
        e1, x1, a0 = h.new_vec(), h.new_vec(), h.new_vec()
        h.lddmm_jacobi_forward(dev(d, dtype), e1, x1)
        h.lddmm_jacobi_adjoint(dev(be, dtype), dev(bx, dtype), a0)
        h.lddmm_synchronize()
    assert rel(host(e1), eta) < tol and rel(host(x1), xi) < tol
    assert rel(host(a0), adj) < tol
    # the GPU sweeps are exact transposes of each other
    lhs = np.sum(host(e1) * be) + np.sum(host(x1) * bx)
    rhs = np.sum(d * host(a0))
    assert abs(lhs - rhs) < (1e-12 if prec == "f64" else 1e-5) * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_jacobian_det(pkg, prec):
    dtype, _ = DT[prec]
    n = (20, 12, 18)
    g = O.Grid(n)
    u = synth.band_limited_field(n, synth.rng_for(11), 3.0, 3) * 0.3 * g.h[0]
    J = O.jacobian_det(g, u)
    with pkg.Handle(n, params(pkg, prec)) as h:
        Jd = h.new_img()
        mm = h.lddmm_jacobian_det(dev(u, dtype), Jd)
    tol = F64_TOL if prec == "f64" else 1e-4
    assert rel(host(Jd) - 1.0, J - 1.0) < tol
    assert abs(mm[0] - J.min()) < tol and abs(mm[1] - J.max()) < tol


@pytest.mark.parametrize("interp", ["cubic", "linear"])
def test_register_replays_oracle(pkg, interp):
    """Whole registration: the FP64 GPU run and the oracle make the same
    decisions (PCG iterations, Armijo steps) and reach the same v0."""
    n = (16, 12, 10)
    nt = 4
    g, I0, I1, vtrue = problem(n, 12, nt)
    p = O.Params(nt=nt, interp=interp)
    kind = pkg.LDDMM_INTERP_CUBIC if interp == "cubic" else pkg.LDDMM_INTERP_LINEAR
    with pkg.Handle(n, params(pkg, "f64", nt=nt, interp=kind, gn_maxit=3, pcg_maxit=6)) as h:
        v = torch.zeros((3,) + n, dtype=torch.float64, device="cuda")
        rep = h.lddmm_register(dev(I0, torch.float64), dev(I1, torch.float64), v)
    ref = O.register(g, p, I0, I1, gn_maxit=3, pcg_maxit=6)
    assert rep["pcg_iters"] == ref.pcg_iters and rep["step"] == ref.steps
    assert rel(host(v), ref.v0) < 1e-9
    assert np.allclose(rep["energy"], ref.energies, rtol=1e-9)
    assert abs(rep["mse_rel"] - ref.mse_rel) < 1e-9 and abs(rep["jac_min"] - ref.jac_min) < 1e-9


def test_register_gradient_descent_matches_oracle(pkg):
    """Gradient descent in V (optimizer LDDMM_OPT_GD): the FP64 GPU run takes
    the oracle's Armijo steps and reaches its v0."""
    n = (16, 12, 10)
    nt = 4
    g, I0, I1, vtrue = problem(n, 12, nt)
    p = O.Params(nt=nt)
    with pkg.Handle(n, params(pkg, "f64", nt=nt, gn_maxit=6, optimizer=pkg.LDDMM_OPT_GD)) as h:
        v = torch.zeros((3,) + n, dtype=torch.float64, device="cuda")
        rep = h.lddmm_register(dev(I0, torch.float64), dev(I1, torch.float64), v)
    ref = O.register_gd(g, p, I0, I1, maxit=6)
    assert rep["pcg_iters"] == [0] * 6 and rep["pcg_iters_total"] == 0
    assert np.allclose(rep["step"], ref.steps, rtol=1e-9, atol=0)
    assert rel(host(v), ref.v0) < 1e-9
    assert np.allclose(rep["energy"], ref.energies, rtol=1e-9)
    assert abs(rep["mse_rel"] - ref.mse_rel) < 1e-9 and abs(rep["gnorm_rel"] - ref.gnorm_rel) < 1e-9


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["cubic", "linear"])
@pytest.mark.parametrize("n", [(10, 12, 8), (32, 32, 32)])
def test_gradient_discrete_matches_oracle(pkg, prec, kind, n):
    """gradient_mode = LDDMM_GRAD_DISCRETE: the exact gradient of the discrete
    energy (transposed map steps and warp) against the oracle's."""
    dtype, _ = DT[prec]
    nt = 3
    g = O.Grid(n, alpha=0.02)
    I0, vt = synth.blob_pair_inputs(n, 5, kmax=2, max_disp_vox=1.5)
    I0 = synth.spectral_gaussian_smooth(I0, 0.8)
    I1 = O.shoot(g, vt, nt, I0, kind).m1 + 0.01 * synth.rng_for(3).standard_normal(n)
    p = O.Params(alpha=0.02, nt=nt, interp=kind)
    v0 = 0.6 * vt + 0.05 * synth.band_limited_field(n, synth.rng_for(4), 2.0, 3) * g.h[0]
    want, E = O.gradient_exact(g, p, v0, I0, I1)
    ik = pkg.LDDMM_INTERP_CUBIC if kind == "cubic" else pkg.LDDMM_INTERP_LINEAR
    prm = params(pkg, prec, alpha=0.02, nt=nt, interp=ik, space=pkg.LDDMM_SPACE_L2,
                 gradient_mode=pkg.LDDMM_GRAD_DISCRETE)
    with pkg.Handle(n, prm) as h:
        grad = h.new_vec()
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        h.lddmm_synchronize()
        got = host(grad)
    tol = 1e-10 if prec == "f64" else 1e-5
    assert abs(e[0] - E) < tol * E
    assert rel(got, want) < tol, rel(got, want)


@pytest.mark.parametrize("n", [(16, 12, 10), (32, 32, 32)])
def test_register_fp32_form_replayed_in_oracle(pkg, n):
    """Whole registration in the FP32 form: the oracle replays the GPU's
    decisions (PCG iterations and Armijo steps per Gauss-Newton iteration)
    in FP64, and the outcomes agree within the FP32 form's tolerances
    (final residual and Jacobian extrema 1e-4, energies 1e-5)."""
    nt = 4
    g, I0, I1, vtrue = problem(n, 14, nt)
    p = O.Params(nt=nt)
    f32 = torch.float32
    prm = params(pkg, "f32", nt=nt, gn_maxit=3, pcg_maxit=6)
    with pkg.Handle(n, prm) as h:
        v = torch.zeros((3,) + n, dtype=f32, device="cuda")
        rep = h.lddmm_register(dev(I0, f32), dev(I1, f32), v)
        v32 = host(v)
    trace = list(zip(rep["pcg_iters"], rep["step"]))
    ref = O.register(g, p, I0, I1, gn_maxit=3, pcg_maxit=6, replay=trace)
    assert rel(v32, ref.v0) < 1e-4
    assert np.allclose(rep["energy"], ref.energies, rtol=1e-5, atol=0)
    assert abs(rep["mse_rel"] - ref.mse_rel) < 1e-4 * ref.mse_rel
    assert abs(rep["jac_min"] - ref.jac_min) < 1e-4 and abs(rep["jac_max"] - ref.jac_max) < 1e-4


def test_register_with_discrete_gradient_replays_oracle(pkg):
    """Gauss-Newton-Krylov with the exact discrete gradient: the FP64 GPU run
    and the oracle make the same PCG and Armijo decisions and reach the same
    v0."""
    n = (16, 12, 10)
    nt = 4
    g, I0, I1, vtrue = problem(n, 12, nt)
    p = O.Params(nt=nt)
    prm = params(pkg, "f64", nt=nt, gn_maxit=3, pcg_maxit=6, gradient_mode=pkg.LDDMM_GRAD_DISCRETE)
    with pkg.Handle(n, prm) as h:
        v = torch.zeros((3,) + n, dtype=torch.float64, device="cuda")
        rep = h.lddmm_register(dev(I0, torch.float64), dev(I1, torch.float64), v)
    ref = O.register(g, p, I0, I1, gn_maxit=3, pcg_maxit=6, exact_gradient=True)
    assert rep["pcg_iters"] == ref.pcg_iters and rep["step"] == ref.steps
    assert rel(host(v), ref.v0) < 1e-9
    assert np.allclose(rep["energy"], ref.energies, rtol=1e-9)
    assert abs(rep["gnorm_rel"] - ref.gnorm_rel) < 1e-9 and abs(rep["mse_rel"] - ref.mse_rel) < 1e-9


def test_gradient_discrete_finite_differences_on_gpu(pkg):
    """The FP64 GPU exact gradient against central differences of the GPU's own
    energy in rough random directions."""
    n, nt = (12, 10, 8), 3
    g = O.Grid(n, alpha=0.02)
    I0, vt = synth.blob_pair_inputs(n, 6, kmax=2, max_disp_vox=1.5)
    I0 = synth.spectral_gaussian_smooth(I0, 0.8)
    I1 = O.shoot(g, vt, nt, I0).m1
    v0 = 0.5 * vt
    prm = params(pkg, "f64", alpha=0.02, nt=nt, space=pkg.LDDMM_SPACE_L2, gradient_mode=pkg.LDDMM_GRAD_DISCRETE)
    f64 = torch.float64
    with pkg.Handle(n, prm) as h:
        grad, scratch = h.new_vec(), h.new_vec()
        h.lddmm_gradient(dev(v0, f64), dev(I0, f64), dev(I1, f64), grad)
        gnp = host(grad)
        r = synth.rng_for(77)
        for _ in range(3):
            d = r.standard_normal((3,) + n) * g.h[0]
            eps = 1e-5
            ep = h.lddmm_gradient(dev(v0 + eps * d, f64), dev(I0, f64), dev(I1, f64), scratch)[0]
            em = h.lddmm_gradient(dev(v0 - eps * d, f64), dev(I0, f64), dev(I1, f64), scratch)[0]
            fd = (ep - em) / (2 * eps)
            assert abs(g.dot(gnp, d) - fd) < 1e-7 * abs(fd)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [(12, 10, 15), (32, 32, 32)])
def test_degenerate_cases(pkg, prec, n):
    """The method's degenerate cases on the GPU: v0 = 0 is the identity map
    (u1 = 0 and m1 = I0 bit for bit, zero kinetic energy); a constant
    velocity of whole voxels per unit time is a rigid roll of the image; at
    v0 = 0 the tangent sweep gives eta1 = xi1 = P delta (eta constant,
    xi' = eta over unit time)."""
    dtype, _ = DT[prec]
    g = O.Grid(n, alpha=0.01)
    I0 = synth.spectral_gaussian_smooth(synth.blob_phantom(n, synth.rng_for(90)), 1.0)
    I0d = dev(I0, dtype)
    tol = 1e-12 if prec == "f64" else 1e-5
    with pkg.Handle(n, params(pkg, prec, nt=4)) as h:
        m1, u1 = h.new_img(), h.new_vec()
        kin = h.lddmm_shoot(dev(np.zeros((3,) + n), dtype), I0d, m1, u1, kinetic=True)
        h.lddmm_synchronize()
        assert torch.equal(u1, torch.zeros_like(u1))
        assert torch.equal(m1, I0d)
        assert all(k == 0.0 for k in kin)
        # whole-voxel constant velocity: (2, -1, 3) voxels over unit time
        shift = (2, -1, 3)
        vc = np.stack([np.full(n, s * g.h[a]) for a, s in enumerate(shift)])
        h.lddmm_shoot(dev(vc, dtype), I0d, m1, u1)
        h.lddmm_synchronize()
        want = np.roll(I0, shift, axis=(0, 1, 2))
        assert rel(host(m1), want) < tol
        assert rel(host(u1), -vc) < tol
        # sweeps at v0 = 0
        d = synth.band_limited_field(n, synth.rng_for(91), 6.0, 3) + 0.1 * synth.rng_for(92).standard_normal((3,) + n)
        z = dev(np.zeros((3,) + n), dtype)
        h.lddmm_shoot(z, I0d, m1)
        e1, x1 = h.new_vec(), h.new_vec()
        h.lddmm_jacobi_forward(dev(d, dtype), e1, x1)
        h.lddmm_synchronize()
        assert rel(host(e1), g.P(d)) < tol and rel(host(x1), g.P(d)) < tol


MAP_STEP_CASES = [
    # (grid, constant velocity in voxels over unit time, peak of the random part)
    ((12, 10, 15), (0.0, 0.0, 2.0), 2.0),   # the staged box wraps onto itself
    ((32, 32, 32), (0.0, 0.0, 1.0), 4.0),   # about a quarter of the points leave the box
    ((32, 32, 32), (2.0, -2.0, 2.0), 3.0),  # nearly every point leaves the box
]


@pytest.mark.parametrize("interp", ["cubic", "linear"])
@pytest.mark.parametrize("n,shift,peak", MAP_STEP_CASES)
def test_map_step_beyond_staged_box(pkg, interp, n, shift, peak, monkeypatch):
    """Semi-Lagrangian map steps (Sec. 3 state equation, reading C6) whose
    departure points lie more than one voxel away: the FP32 staged kernel
    takes its global-gather fallback for those stencils and its shared-memory
    taps for the others, within one block.  Its maps equal those of the plain
    gather kernel (LDDMM_SL_GATHER=1) bit for bit, and both match the oracle;
    the FP64 engine (gather kernel) matches it to 1e-10."""
    nt = 2
    g = O.Grid(n, alpha=0.01)
    I0 = synth.spectral_gaussian_smooth(synth.blob_phantom(n, synth.rng_for(93)), 1.0)
    v0 = synth.random_velocity(n, synth.rng_for(94), 2, peak) + np.stack(
        [np.full(n, shift[a] * g.h[a]) for a in range(3)])
    # departure displacement of the first step, in voxels: some stencils leave
    # the staged box (|d| > 1), others stay inside it
    d = np.abs(v0 / nt / np.array(g.h).reshape(3, 1, 1, 1)).max(axis=0)
    assert (d > 1.25).any() and (d < 0.9).any() or (d > 1.25).mean() > 0.5
    tr = O.shoot(g, v0, nt, I0, kind=interp)
    code = pkg.LDDMM_INTERP_CUBIC if interp == "cubic" else pkg.LDDMM_INTERP_LINEAR
    out = {}
    for mode in ("staged", "gather"):
        if mode == "gather":
            monkeypatch.setenv("LDDMM_SL_GATHER", "1")
        else:
            monkeypatch.delenv("LDDMM_SL_GATHER", raising=False)
        with pkg.Handle(n, params(pkg, "f32", nt=nt, interp=code)) as h:
            m1, u1 = h.new_img(), h.new_vec()
            h.lddmm_shoot(dev(v0, torch.float32), dev(I0, torch.float32), m1, u1)
            h.lddmm_synchronize()
            out[mode] = (u1.clone(), m1.clone())
    monkeypatch.delenv("LDDMM_SL_GATHER", raising=False)
    assert torch.equal(out["staged"][0], out["gather"][0])
    assert torch.equal(out["staged"][1], out["gather"][1])
    assert rel(host(out["staged"][0]), tr.u) < 1e-5
    assert rel(host(out["staged"][1]), tr.m1) < 1e-5
    with pkg.Handle(n, params(pkg, "f64", nt=nt, interp=code)) as h:
        m1, u1 = h.new_img(), h.new_vec()
        h.lddmm_shoot(dev(v0, torch.float64), dev(I0, torch.float64), m1, u1)
        h.lddmm_synchronize()
        assert rel(host(u1), tr.u) < F64_TOL
        assert rel(host(m1), tr.m1) < F64_TOL


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_nonfinite_inputs_are_reported(pkg, prec):
    """A NaN or an infinity in any array input is found by the device scan
    and returned as LDDMM_ERR_NONFINITE (6) by the call that received it; the
    status is then sticky on the handle.  Clean inputs leave it at 0."""
    dtype, _ = DT[prec]
    n = (12, 10, 15)
    nt = 2
    g, I0, I1, vtrue = problem(n, 3, nt)
    v0 = 0.5 * vtrue
    bad = np.zeros((3,) + n)
    bad[1, 3, 4, 5] = np.nan
    badimg = I1.copy()
    badimg[2, 0, 7] = np.inf

    def linearised():
        h = pkg.Handle(n, params(pkg, prec, nt=nt))
        h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), h.new_vec())
        return h

    calls = [
        ("hessvec", lambda h: h.lddmm_hessvec(dev(bad, dtype), h.new_vec())),
        ("jacobi_forward", lambda h: h.lddmm_jacobi_forward(dev(bad, dtype), h.new_vec(), h.new_vec())),
        ("jacobi_adjoint", lambda h: h.lddmm_jacobi_adjoint(None, dev(bad, dtype), h.new_vec())),
        ("shoot_vjp", lambda h: h.lddmm_shoot_vjp(dev(badimg, dtype), h.new_vec())),
        ("shoot", lambda h: h.lddmm_shoot(dev(bad + v0, dtype), dev(I0, dtype), h.new_img())),
        ("gradient", lambda h: h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(badimg, dtype), h.new_vec())),
        ("apply_metric", lambda h: h.lddmm_apply_metric(dev(bad, dtype), h.new_vec(), -1)),
        ("jacobian_det", lambda h: h.lddmm_jacobian_det(dev(bad, dtype))),
        ("register", lambda h: h.lddmm_register(dev(I0, dtype), dev(badimg, dtype), dev(np.zeros((3,) + n), dtype))),
    ]
    for name, call in calls:
        with linearised() as h:
            assert pkg.lib().lddmm_last_status(h._h) == 0, name
            with pytest.raises(pkg.LddmmError) as ei:
                call(h)
                h.lddmm_synchronize()
            assert ei.value.status == 6, (name, ei.value.status)
            # sticky: a clean call on the same handle reports it again
            with pytest.raises(pkg.LddmmError) as ei:
                h.lddmm_hessvec(dev(v0, dtype), h.new_vec())
            assert ei.value.status == 6, name
    # clean inputs: no false alarm, also after a run of calls
    with linearised() as h:
        out = h.new_vec()
        for _ in range(3):
            h.lddmm_hessvec(dev(v0, dtype), out)
        h.lddmm_apply_metric(dev(v0, dtype), out, 1)
        h.lddmm_synchronize()
        assert pkg.lib().lddmm_last_status(h._h) == 0


def test_errors_are_reported(pkg):
    n = (8, 8, 8)
    with pytest.raises(pkg.LddmmError):
        pkg.Handle((7, 8, 8), pkg.default_params())
    with pkg.Handle(n, pkg.default_params()) as h:
        out = h.new_vec()
        with pytest.raises(pkg.LddmmError) as ei:
            h.lddmm_hessvec(torch.zeros((3,) + n, dtype=torch.float64, device="cuda"), out)
        assert ei.value.status == 5
        with pytest.raises(TypeError):
            h.lddmm_shoot(torch.zeros((3,) + n, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_unfiltered_products_option(pkg, prec):
    """dealias = 0 reproduces the literal unfiltered scheme of the oracle."""
    dtype, _ = DT[prec]
    n = (20, 12, 18)
    nt = 4
    g = O.Grid(n, alpha=0.01, dealias=False)
    I0, vtrue = synth.blob_pair_inputs(n, 6, kmax=2, max_disp_vox=1.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, nt, I0).m1
    p = O.Params(nt=nt)
    v0 = 0.5 * vtrue
    gl2, E, _, _, tr = O.gradient(g, p, v0, I0, I1)
    d = synth.band_limited_field(n, synth.rng_for(8), 4.0, 3) * g.h[0]
    hl2 = O.hessvec(g, p, tr, d)
    tol = F64_TOL if prec == "f64" else 1e-5
    with pkg.Handle(n, params(pkg, prec, nt=nt, dealias=0)) as h:
        grad, hv = h.new_vec(), h.new_vec()
        e = h.lddmm_gradient(dev(v0, dtype), dev(I0, dtype), dev(I1, dtype), grad)
        h.lddmm_hessvec(dev(d, dtype), hv)
        h.lddmm_synchronize()
    assert abs(e[0] - E) < tol * abs(E)
    assert rel(host(grad), O.to_space(g, p, gl2)) < tol
    assert rel(host(hv), O.to_space(g, p, hl2)) < tol


def test_fp64_fma_probe(pkg):
    """The FP64 rate probe runs, writes finite values and reports a rate
    within loose sanity bounds (not a performance assertion)."""
    tf = pkg.probe_fp64_fma(iters=256, reps=2)
    assert 0.01 < tf < 200.0
