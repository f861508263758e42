"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, conservation laws of the EPDiff equation, exact discrete transposes,
finite differences, special cases that reduce to textbook results, and brute
force on tiny grids.  None of them needs a GPU.
"""
import math

import numpy as np
import pytest

from oracle import lddmm_oracle as O
from paper_1807_04638_gb300 import synth

TWO_PI = 2 * math.pi


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def band(n, seed, kmax, ncomp=3, scale=1.0):
    return scale * synth.band_limited_field(n, synth.rng_for(seed), kmax, ncomp)


def rough(n, seed, ncomp=3):
    r = synth.rng_for(seed)
    return r.standard_normal((ncomp,) + tuple(n)) if ncomp > 1 else r.standard_normal(tuple(n))


def phys(g):
    return [g.coords[a] * g.h[a] for a in range(3)]


# --------------------------------------------------------------------------
# Spectral operators (Sec. 2.1 metric; pseudo-spectral derivatives)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,lengths", [((8, 12, 10), None), ((6, 10, 16), (1.0, 2.5, 4.0))])
def test_derivative_closed_form(n, lengths):
    g = O.Grid(n, lengths=lengths)
    x = phys(g)
    for a in range(3):
        k = 2
        w = TWO_PI * k / g.lengths[a]
        f = np.sin(w * x[a] + 0.3)
        assert rel(g.D(f, a), w * np.cos(w * x[a] + 0.3)) < 1e-13
        # other axes see a constant along themselves
        for b in range(3):
            if b != a:
                assert np.abs(g.D(f, b)).max() < 1e-13


def test_derivative_nyquist_is_zeroed():
    g = O.Grid((8, 6, 10))
    for a in range(3):
        f = np.cos(math.pi * g.coords[a])  # the Nyquist mode along axis a
        assert np.abs(g.D(f, a)).max() < 1e-13


def test_K_of_fourier_mode_closed_form():
    g = O.Grid((8, 12, 10), alpha=0.05, s=2, lengths=(1.0, 2.0, 3.0))
    x = phys(g)
    kv = (1, -2, 3)
    kap = [TWO_PI * kv[a] / g.lengths[a] for a in range(3)]
    f = np.cos(sum(kap[a] * x[a] for a in range(3)))
    lam = (1 + g.alpha * sum(k * k for k in kap)) ** g.s
    assert rel(g.K(f), f / lam) < 1e-13
    assert rel(g.L(f), f * lam) < 1e-13


def test_K_inverts_L_and_D_is_skew():
    g = O.Grid((8, 6, 10), alpha=0.02, s=2)
    f, h = rough(g.n, 1, 1), rough(g.n, 2, 1)
    assert rel(g.K(g.L(f)), f) < 1e-13
    for a in range(3):
        lhs = g.dot(g.D(f, a), h)
        rhs = -g.dot(f, g.D(h, a))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # K and L are symmetric
    assert abs(g.dot(g.K(f), h) - g.dot(f, g.K(h))) < 1e-13 * abs(g.dot(g.K(f), h))


# --------------------------------------------------------------------------
# ad* and ad (Sec. 2.2 EPDiff bracket)
# --------------------------------------------------------------------------

def test_ad_star_closed_form_single_mode():
    """v = a sin(k.x), m = b constant:  ad*_v m = k (a.b) cos + b (k.a) cos.
    v = c constant, m = b sin(k.x):     ad*_v m = (k.c) b cos."""
    g = O.Grid((8, 10, 12), lengths=(2.0, 3.0, 4.0))
    x = phys(g)
    kv = (1, 2, -1)
    kap = np.array([TWO_PI * kv[a] / g.lengths[a] for a in range(3)])
    ph = sum(kap[a] * x[a] for a in range(3))
    a = np.array([0.3, -0.7, 0.5])
    b = np.array([1.1, 0.4, -0.9])
    v = a.reshape(3, 1, 1, 1) * np.sin(ph)
    m = b.reshape(3, 1, 1, 1) * np.ones(g.n)
    want = (kap * (a @ b) + b * (kap @ a)).reshape(3, 1, 1, 1) * np.cos(ph)
    assert rel(O.ad_star(g, v, m), want) < 1e-13
    c = np.array([0.2, 0.6, -0.3])
    v = c.reshape(3, 1, 1, 1) * np.ones(g.n)
    m = b.reshape(3, 1, 1, 1) * np.sin(ph)
    want = (kap @ c) * b.reshape(3, 1, 1, 1) * np.cos(ph)
    assert rel(O.ad_star(g, v, m), want) < 1e-13


def test_ad_closed_form_and_antisymmetry():
    """ad_c w for constant c: -(Dw) c = -(k.c) b cos for w = b sin(k.x)."""
    g = O.Grid((8, 10, 12))
    x = phys(g)
    kap = np.array([1.0, 2.0, -1.0])
    ph = sum(kap[a] * x[a] for a in range(3))
    b = np.array([1.1, 0.4, -0.9])
    c = np.array([0.2, 0.6, -0.3])
    w = b.reshape(3, 1, 1, 1) * np.sin(ph)
    cv = c.reshape(3, 1, 1, 1) * np.ones(g.n)
    assert rel(O.ad(g, cv, w), -(kap @ c) * b.reshape(3, 1, 1, 1) * np.cos(ph)) < 1e-13
    v, u = rough(g.n, 3), rough(g.n, 4)
    assert rel(O.ad(g, v, u), -O.ad(g, u, v)) < 1e-13
    assert np.abs(O.ad(g, v, v)).max() < 1e-12


def test_ad_star_is_dual_of_ad_when_products_resolve():
    g = O.Grid((12, 12, 12))
    v, m, w = band(g.n, 5, 2.0), band(g.n, 6, 2.0), band(g.n, 7, 2.0)
    lhs = g.dot(O.ad_star(g, v, m), w)
    rhs = g.dot(m, O.ad(g, v, w))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_dealiased_products_are_exact():
    """With the 2/3 rule, P ad*_v m is dual to P ad_v P exactly for any
    band-limited v, m, w (all quadratic products resolved), and the energy
    rate <L v, R(v)> vanishes for every band-limited v, not only for the
    small band where unfiltered products resolve."""
    g = O.Grid((12, 12, 12), alpha=0.02)
    r = synth.rng_for(17)
    v, m, w = (g.P(r.standard_normal((3,) + g.n)) for _ in range(3))
    lhs = g.dot(g.P(O.ad_star(g, v, m)), w)
    rhs = g.dot(m, g.P(O.ad(g, v, w)))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + abs(rhs))
    rr = O.epdiff_rhs(g, v)
    assert abs(g.dot(g.L(v), rr)) < 1e-12 * math.sqrt(g.dot(rr, rr) * g.dot(g.L(v), g.L(v)))
    # the filtered right-hand side stays in the band; the unfiltered one leaves it
    assert rel(g.P(rr), rr) < 1e-14
    r0 = O.epdiff_rhs(O.Grid((12, 12, 12), alpha=0.02, dealias=False), v)
    assert rel(g.P(r0), r0) > 1e-3


def test_epdiff_rhs_conserves_energy_and_momentum():
    """d/dt <Lv, v> = -2 <ad*_v Lv, v> = 0 and d/dt mean(v) = 0 (EPDiff
    invariants), exactly for band-limited v whose products resolve."""
    g = O.Grid((12, 12, 12), alpha=0.02)
    v = band(g.n, 8, 2.0)
    r = O.epdiff_rhs(g, v)
    assert abs(g.dot(g.L(v), r)) < 1e-12 * np.linalg.norm(r) * np.linalg.norm(v) * g.cell
    assert np.abs(r.mean(axis=(1, 2, 3))).max() < 1e-14 * np.abs(r).max()


# --------------------------------------------------------------------------
# Exact discrete transposes (dot-product tests)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [(6, 8, 10), (5, 6, 9)])
def test_transposes_dot_tests(n):
    g = O.Grid(n, alpha=0.03)
    v, m, x, y = rough(n, 10), rough(n, 11), rough(n, 12), rough(n, 13)

    def check(fwd, tr):
        a = g.dot(fwd(x), y)
        b = g.dot(x, tr(y))
        assert abs(a - b) < 1e-12 * (abs(a) + abs(b)), (a, b)

    check(lambda e: O.ad_star(g, e, m), lambda z: O.ad_star_T_first(g, m, z))
    check(lambda e: O.ad_star(g, v, e), lambda z: O.ad_star_T_second(g, v, z))
    check(lambda e: O.ad(g, v, e), lambda z: O.ad_T(g, v, z))
    check(lambda e: O.epdiff_rhs_lin(g, v, e), lambda z: O.epdiff_rhs_lin_T(g, v, z))
    x2, y2 = rough(n, 14), rough(n, 15)
    fa, fb = O.jacobi_A(g, v, x, x2)
    ta, tb = O.jacobi_A_T(g, v, y, y2)
    a = g.dot(fa, y) + g.dot(fb, y2)
    b = g.dot(x, ta) + g.dot(x2, tb)
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))


# --------------------------------------------------------------------------
# Shooting (EPDiff, Heun)
# --------------------------------------------------------------------------

def test_shoot_zero_velocity_is_identity():
    g = O.Grid((8, 10, 6))
    I0 = rough(g.n, 20, 1)
    tr = O.shoot(g, np.zeros((3,) + g.n), 5, I0)
    assert all(np.abs(v).max() == 0 for v in tr.v)
    assert np.abs(tr.u).max() == 0
    assert np.array_equal(tr.m1, I0)


def test_shoot_constant_velocity():
    """Constant v0: ad* vanishes, v_t = v0, u_1 = -v0, and an integer-voxel
    v0 makes m(1) a periodic roll of I0."""
    g = O.Grid((8, 10, 12))
    c = np.array([2 * g.h[0], -1 * g.h[1], 3 * g.h[2]])
    v0 = c.reshape(3, 1, 1, 1) * np.ones(g.n)
    I0 = rough(g.n, 21, 1)
    for kind in ("cubic", "linear"):
        tr = O.shoot(g, v0, 10, I0, kind)
        assert rel(tr.v[-1], v0) < 1e-14
        assert rel(tr.u, -v0) < 1e-13
        assert rel(tr.m1, np.roll(I0, shift=(2, -1, 3), axis=(0, 1, 2))) < 1e-12


def test_shoot_momentum_and_energy_convergence():
    """Mean of v (linear momentum, K_hat(0) = 1) is conserved exactly.  The
    kinetic energy <L v_t, v_t> is an invariant of the EPDiff flow and, with
    dealiased products, of the semi-discrete scheme too: the Heun drift goes
    to zero at least at second order in dt."""
    g = O.Grid((16, 16, 16), alpha=0.01)
    v0 = synth.random_velocity(g.n, synth.rng_for(3), 2.0, 1.0)
    drifts = []
    for nt in (5, 10, 20, 40):
        tr = O.shoot(g, v0, nt)
        assert np.abs(tr.v[-1].mean(axis=(1, 2, 3)) - v0.mean(axis=(1, 2, 3))).max() < 1e-13
        drifts.append(abs(tr.kinetic[-1] - tr.kinetic[0]) / tr.kinetic[0])
    assert drifts[-1] < 1e-6, drifts
    for a, b in zip(drifts, drifts[1:]):
        assert a / b > 3.5, drifts


def test_tangent_is_exact_linearisation_of_discrete_shooting():
    g = O.Grid((8, 8, 8), alpha=0.02)
    v0 = synth.random_velocity(g.n, synth.rng_for(4), 2.0, 1.5)
    d = band(g.n, 30, 2.0, scale=0.1)
    nt = 4
    tr = O.shoot(g, v0, nt)
    eta, _ = O.tangent(g, tr, d)
    eps = 1e-5
    fd = (O.shoot(g, v0 + eps * d, nt).v[-1] - O.shoot(g, v0 - eps * d, nt).v[-1]) / (2 * eps)
    assert rel(eta, fd) < 1e-8


def test_tangent_constant_background_matches_heun_matrix_polynomial():
    """v_t = c constant, dv0 = a sin(k.x) + b cos(k.x): each Fourier mode obeys a
    6x6 constant-coefficient linear ODE whose Heun step is I + dt A + dt^2 A^2/2."""
    g = O.Grid((8, 8, 8), alpha=0.05, s=2)
    x = phys(g)
    kap = np.array([1.0, -2.0, 1.0])
    c = np.array([0.4, -0.3, 0.7])
    a = np.array([0.2, 0.5, -0.4])
    b = np.array([-0.1, 0.3, 0.6])
    ph = sum(kap[i] * x[i] for i in range(3))
    d = a.reshape(3, 1, 1, 1) * np.sin(ph) + b.reshape(3, 1, 1, 1) * np.cos(ph)
    nt = 7
    tr = O.shoot(g, c.reshape(3, 1, 1, 1) * np.ones(g.n), nt)
    eta, xi = O.tangent(g, tr, d)
    # complex amplitude: field = Re(A e^{i k.x}) with A = b - i a
    lam = (1 + g.alpha * kap @ kap) ** g.s
    kc = kap @ c
    # eta' = -K [ (D eta)^T c + c div eta + (D L eta) c ]   on a mode: i(...)
    Mee = -1j / lam * (np.outer(kap, c) + np.outer(c, kap) + lam * kc * np.eye(3))
    A = np.zeros((6, 6), complex)
    A[:3, :3] = Mee
    A[3:, :3] = np.eye(3)
    A[3:, 3:] = -1j * kc * np.eye(3)          # xi' = eta + ad_c xi = eta - (D xi) c
    dt = 1.0 / nt
    step = np.eye(6) + dt * A + 0.5 * dt * dt * A @ A
    z = np.linalg.matrix_power(step, nt) @ np.concatenate([b - 1j * a, np.zeros(3)])
    want_eta = (z[:3].reshape(3, 1, 1, 1) * np.exp(1j * ph)).real
    want_xi = (z[3:].reshape(3, 1, 1, 1) * np.exp(1j * ph)).real
    assert rel(eta, want_eta) < 1e-12
    assert rel(xi, want_xi) < 1e-12


# --------------------------------------------------------------------------
# Interpolation and semi-Lagrangian transport
# --------------------------------------------------------------------------

def test_interp_polynomial_reproduction():
    """Trilinear reproduces affine data, Catmull-Rom quadratics (away from the
    periodic seam, where the samples are that polynomial)."""
    n = (16, 16, 16)
    i = np.stack(np.meshgrid(*[np.arange(m, dtype=float) for m in n], indexing="ij"))
    r = synth.rng_for(40)
    p = 4.0 + 7.0 * r.random((3, 200))
    aff = lambda q: 0.3 + 0.2 * q[0] - 0.7 * q[1] + 0.05 * q[2]
    quad = lambda q: 0.1 + 0.02 * q[0] ** 2 - 0.03 * q[1] * q[2] + 0.01 * q[2] ** 2 + 0.2 * q[0]
    assert np.abs(O.interp(aff(i), p, "linear") - aff(p)).max() < 1e-12
    assert np.abs(O.interp(quad(i), p, "cubic") - quad(p)).max() < 1e-12
    # interpolating: integer coordinates return samples (with wrap)
    f = r.standard_normal(n)
    q = np.stack([i[a] + s for a, s in enumerate((3, -5, 17))])
    for kind in ("linear", "cubic"):
        assert np.array_equal(O.interp(f, q, kind), np.roll(f, (-3, 5, -17), (0, 1, 2)))


def test_sl_constant_noninteger_velocity():
    g = O.Grid((12, 10, 8))
    c = np.array([0.37 * g.h[0], -1.3 * g.h[1], 0.81 * g.h[2]])
    v0 = c.reshape(3, 1, 1, 1) * np.ones(g.n)
    I0 = rough(g.n, 41, 1)
    tr = O.shoot(g, v0, 6, I0)
    assert rel(tr.u, -v0) < 1e-13
    want = O.interp(I0, g.coords - (c / np.array(g.h)).reshape(3, 1, 1, 1), "cubic")
    assert rel(tr.m1, want) < 1e-12


def test_jacobian_det_closed_form_and_null_lagrangian():
    g = O.Grid((12, 12, 12))
    x = phys(g)
    kap = np.array([1.0, 2.0, 0.0])
    a = np.array([0.05, 0.1, -0.2])
    ph = sum(kap[i] * x[i] for i in range(3))
    u = a.reshape(3, 1, 1, 1) * np.sin(ph)
    assert np.abs(O.jacobian_det(g, u) - (1 + (kap @ a) * np.cos(ph))).max() < 1e-13
    u = band(g.n, 42, 2.0, scale=0.05)
    assert abs(O.jacobian_det(g, u).mean() - 1.0) < 1e-13


# --------------------------------------------------------------------------
# Jacobi sweeps, gradient and Gauss-Newton Hessian (Sec. 3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dealias", [True, False])
def test_sweeps_at_zero_velocity_are_the_projector(dealias):
    """At v = 0: eta stays P dv0 and xi_nt = sum dt P dv0 = P dv0; T^T = P."""
    g = O.Grid((6, 8, 6), dealias=dealias)
    tr = O.shoot(g, np.zeros((3,) + g.n), 6)
    d = rough(g.n, 50)
    Pd = g.P(d)
    eta, xi = O.tangent(g, tr, d)
    assert rel(eta, Pd) < 1e-14 and rel(xi, Pd) < 1e-14
    assert rel(O.adjoint(g, tr, d), Pd) < 1e-14
    if not dealias:
        assert rel(Pd, d) < 1e-15


def test_sweep_dot_test():
    g = O.Grid((6, 8, 10), alpha=0.03)
    v0 = synth.random_velocity(g.n, synth.rng_for(51), 2.0, 1.0)
    tr = O.shoot(g, v0, 5)
    d, ye, yx = rough(g.n, 52), rough(g.n, 53), rough(g.n, 54)
    eta, xi = O.tangent(g, tr, d)
    a = g.dot(eta, ye) + g.dot(xi, yx)
    b = g.dot(d, O.adjoint(g, tr, yx, ye))
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))


def test_gradient_and_hessian_closed_form_at_zero():
    g = O.Grid((8, 6, 10), alpha=0.02)
    p = O.Params(alpha=0.02, nt=5)
    I0 = synth.blob_phantom(g.n, synth.rng_for(60), nblobs=3, sigma_vox=(1.0, 2.0))
    I1 = synth.blob_phantom(g.n, synth.rng_for(61), nblobs=3, sigma_vox=(1.0, 2.0))
    zero = np.zeros((3,) + g.n)
    gl2, E, data, reg, tr = O.gradient(g, p, zero, I0, I1)
    gI0 = g.grad(I0)
    assert rel(gl2, g.P(-2 * (I0 - I1)[None] * gI0)) < 1e-13
    assert reg == 0.0 and abs(data - g.dot(I0 - I1, I0 - I1)) < 1e-14
    d = rough(g.n, 62)
    want = 2 * p.weight * g.L(d) + g.P(2 * np.sum(gI0 * g.P(d), 0)[None] * gI0)
    assert rel(O.hessvec(g, p, tr, d), want) < 1e-13


def _small_problem(n=(4, 4, 4), seed=70, nt=4):
    g = O.Grid(n, alpha=0.05)
    p = O.Params(alpha=0.05, nt=nt, weight=1e-2)
    r = synth.rng_for(seed)
    I0 = synth.spectral_gaussian_smooth(r.standard_normal(n), 0.6)
    I1 = synth.spectral_gaussian_smooth(r.standard_normal(n), 0.6)
    v0 = 0.3 * synth.spectral_gaussian_smooth(r.standard_normal(n), 0.6)[None] * np.array(
        [1.0, -0.5, 0.8]).reshape(3, 1, 1, 1)
    return g, p, I0, I1, v0


def _dense_hessian(g, p, tr):
    m = 3 * int(np.prod(g.n))
    H = np.empty((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        H[:, j] = O.hessvec(g, p, tr, e.reshape((3,) + g.n)).ravel()
    return H


@pytest.mark.parametrize("n", [(4, 4, 4), (4, 6, 4)])
def test_dense_gauss_newton_hessian_symmetric_positive(n):
    g, p, I0, I1, v0 = _small_problem(n)
    tr = O.gradient(g, p, v0, I0, I1)[4]
    H = _dense_hessian(g, p, tr)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    # 2 w L >= 2 w (L_hat >= 1) and T^T M T >= 0
    assert ev.min() >= 2 * p.weight * (1 - 1e-10)


def test_pcg_reaches_dense_solve():
    g, p, I0, I1, v0 = _small_problem()
    gl2, _, _, _, tr = O.gradient(g, p, v0, I0, I1)
    H = _dense_hessian(g, p, tr)
    x_ref = np.linalg.solve(H, -gl2.ravel()).reshape(gl2.shape)
    x, it = O.pcg(g, lambda d: O.hessvec(g, p, tr, d), -gl2, g.K, 400, 1e-13)
    assert rel(x, x_ref) < 1e-9


def test_gradient_matches_finite_differences_up_to_linearisation_gap():
    """The Jacobi-field gradient linearises m(1) through -grad m(1) . xi(1),
    not through the interpolation stencil of the semi-Lagrangian transport,
    so it agrees with central differences of the discrete energy only up to
    a discretisation gap that shrinks when h and dt are refined together
    (about 1e-2 of |g||d| at 12^3 / nt = 4, under 2e-3 at 24^3 / nt = 8)."""
    worst = {}
    for n, nt in ((12, 4), (24, 8)):
        g = O.Grid((n, n, n), alpha=0.01)
        I0, vtrue = synth.blob_pair_inputs(g.n, 80, kmax=2, max_disp_vox=n / 12)
        I0 = synth.spectral_gaussian_smooth(I0, 1.5 * n / 12)
        p = O.Params(nt=nt)
        I1 = O.shoot(g, vtrue, 8, I0).m1
        v0 = 0.5 * vtrue
        gl2 = O.gradient(g, p, v0, I0, I1)[0]
        dirs = [gl2 / math.sqrt(g.dot(gl2, gl2)) * g.h[0]]
        dirs += [band(g.n, 90 + s, 2.0, scale=g.h[0]) for s in range(2)]
        worst[n] = 0.0
        for d in dirs:
            eps = 1e-4
            fd = (O.energy(g, p, v0 + eps * d, I0, I1)[0]
                  - O.energy(g, p, v0 - eps * d, I0, I1)[0]) / (2 * eps)
            gd = g.dot(gl2, d)
            worst[n] = max(worst[n], abs(gd - fd) / math.sqrt(g.dot(gl2, gl2) * g.dot(d, d)))
    # the gap is small and shrinks under joint refinement of h and dt
    assert worst[12] < 3e-2 and worst[24] < 5e-3 and worst[24] < 0.3 * worst[12], worst


def test_gauss_newton_decreases_energy_and_replays():
    g = O.Grid((8, 8, 8), alpha=0.02)
    p = O.Params(alpha=0.02, nt=4, weight=1e-3)
    I0, vtrue = synth.blob_pair_inputs(g.n, 95, kmax=2, max_disp_vox=1.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, p.nt, I0).m1
    rep = O.register(g, p, I0, I1, gn_maxit=3, pcg_maxit=5)
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rep.mse_rel < 0.5 and rep.jac_min > 0
    again = O.register(g, p, I0, I1, gn_maxit=3, pcg_maxit=5,
                       replay=list(zip(rep.pcg_iters, rep.steps)))
    assert rel(again.v0, rep.v0) < 1e-14


def test_gradient_descent_in_V_steps_and_armijo():
    """Gradient descent in V (Sec. 2.2): every accepted step moves along
    -K g_L2 with g_L2 the reduced gradient, satisfies the Armijo condition
    recomputed from the energy, decreases E; the first trial step moves
    max |K g| by one voxel, so the first accepted step is that times 2^-k;
    a replay reproduces the iterates."""
    g = O.Grid((8, 8, 8), alpha=0.02)
    p = O.Params(alpha=0.02, nt=4, weight=1e-3)
    I0, vtrue = synth.blob_pair_inputs(g.n, 96, kmax=2, max_disp_vox=1.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, p.nt, I0).m1
    rep = O.register_gd(g, p, I0, I1, maxit=4)
    assert all(b < a for a, b in zip(rep.energies, rep.energies[1:]))
    assert rep.pcg_iters == [0] * len(rep.steps)
    # first step: h / max|K g(0)| halved an integer number of times; at v0 = 0
    # the gradient is the closed form P(-2 (I0 - I1) grad I0)
    g0 = g.P(-2.0 * (I0 - I1)[None] * g.grad(I0))
    k0 = float(np.abs(g.K(g0)).max())
    ratio = rep.steps[0] / (min(g.h) / k0)
    assert abs(np.log2(ratio) - round(np.log2(ratio))) < 1e-9 and ratio <= 1.0
    # replay the steps one at a time and check Armijo along -K g_L2
    v = np.zeros((3,) + g.n)
    for eps in rep.steps:
        gl2, E = O.gradient(g, p, v, I0, I1)[:2]
        x = -g.K(gl2)
        Et = O.energy(g, p, v + eps * x, I0, I1)[0]
        assert Et <= E + 1e-4 * eps * g.dot(gl2, x)
        v = v + eps * x
    assert rel(v, rep.v0) < 1e-14
    again = O.register_gd(g, p, I0, I1, maxit=4, replay=rep.steps)
    assert rel(again.v0, rep.v0) < 1e-14


def _delta_m_routes(n, nt, kind):
    """delta m(1) by the literal incremental state equation and by
    -grad m(1) . xi(1), for smooth inputs fixed in physical coordinates."""
    g = O.Grid((n, n, n), alpha=0.01)
    x = phys(g)
    I0 = np.exp(np.cos(x[0]) + 0.5 * np.sin(x[1]) * np.cos(x[2]))
    v0 = 0.4 * np.stack([np.sin(x[1]), np.sin(x[2]), np.sin(x[0])])
    d = 0.3 * np.stack([np.cos(x[2]), np.cos(x[0] + x[1]), np.sin(x[1])])
    tr = O.shoot(g, v0, nt, I0, kind)
    etas, xi = O.tangent_path(g, tr, d)
    assert rel(xi, O.tangent(g, tr, d)[1]) < 1e-14
    lit = O.incremental_state_literal(g, tr, I0, etas, kind)
    return rel(lit, -np.sum(tr.grad_m1 * xi, axis=0))


def test_incremental_state_equation_agrees_with_jacobi_field_route():
    """The paper's incremental state equation (Sec. 3), integrated along the
    characteristics, and delta m(1) = -grad m(1) . xi(1) (the route the sweeps
    use) approximate the same continuum quantity: their gap shrinks under
    joint refinement of h and dt, at second order with Catmull-Rom and first
    order with trilinear interpolation."""
    e16, e32 = _delta_m_routes(16, 4, "cubic"), _delta_m_routes(32, 8, "cubic")
    assert e32 < 0.01 and e32 < 0.35 * e16, (e16, e32)
    l16, l32 = _delta_m_routes(16, 4, "linear"), _delta_m_routes(32, 8, "linear")
    assert l32 < 0.05 and l32 < 0.65 * l16, (l16, l32)


@pytest.mark.parametrize("kind", ["cubic", "linear"])
def test_interp_transpose_and_coordinate_derivative(kind):
    """The scatter interp_T is the exact transpose of interp (dot test), and
    interp_grad is the derivative of interp with respect to the coordinates
    (central differences)."""
    n = (7, 6, 9)
    r = synth.rng_for(120)
    f = r.standard_normal((2,) + n)
    pts = r.uniform(-3.0, 12.0, (3, 5, 4, 6))
    y = r.standard_normal((2, 5, 4, 6))
    lhs = float(np.sum(O.interp(f, pts, kind) * y))
    rhs = float(np.sum(f * O.interp_T(y, pts, n, kind)))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + abs(rhs))
    G = O.interp_grad(f, pts, kind)
    for a in range(3):
        e = np.zeros((3, 1, 1, 1))
        e[a] = 1e-6
        fd = (O.interp(f, pts + e, kind) - O.interp(f, pts - e, kind)) / 2e-6
        assert rel(G[a], fd) < 1e-7


@pytest.mark.parametrize("kind", ["cubic", "linear"])
def test_exact_discrete_gradient_matches_finite_differences(kind):
    """With the semi-Lagrangian steps and the warp transposed exactly, the
    gradient is the derivative of the discrete energy: central differences in
    random (rough) directions agree to 1e-7 (the Jacobi-field gradient of
    Sec. 3 differs from them by its linearisation gap, order one on this
    coarse grid)."""
    n, nt = (10, 12, 8), 3
    g = O.Grid(n, alpha=0.02)
    I0, vt = synth.blob_pair_inputs(n, 5, kmax=2, max_disp_vox=1.5)
    I0 = synth.spectral_gaussian_smooth(I0, 0.8)
    I1 = O.shoot(g, vt, nt, I0, kind).m1 + 0.01 * synth.rng_for(3).standard_normal(n)
    p = O.Params(alpha=0.02, nt=nt, interp=kind)
    v0 = 0.6 * vt + 0.05 * synth.band_limited_field(n, synth.rng_for(4), 2.0, 3) * g.h[0]
    ge, E = O.gradient_exact(g, p, v0, I0, I1)
    assert abs(E - O.energy(g, p, v0, I0, I1)[0]) < 1e-15 * E
    r = synth.rng_for(9)
    for _ in range(4):
        d = r.standard_normal((3,) + n) * g.h[0]
        eps = 1e-5
        fd = (O.energy(g, p, v0 + eps * d, I0, I1)[0] - O.energy(g, p, v0 - eps * d, I0, I1)[0]) / (2 * eps)
        assert abs(g.dot(ge, d) - fd) < 1e-7 * abs(fd)
    # closed form at v0 = 0: the map moves by -P delta, and the warp's
    # derivative at the grid nodes is the interpolant's own finite difference
    # (central for Catmull-Rom, forward for trilinear), so
    # g = P(-2 (I0 - I1) D_h I0) with that difference in place of grad
    zero = np.zeros((3,) + n)
    if kind == "cubic":
        Dh = [(np.roll(I0, -1, a) - np.roll(I0, 1, a)) / (2 * g.h[a]) for a in range(3)]
    else:
        Dh = [(np.roll(I0, -1, a) - I0) / g.h[a] for a in range(3)]
    want = g.P(-2.0 * (I0 - I1)[None] * np.stack(Dh))
    assert rel(O.gradient_exact(g, p, zero, I0, I1)[0], want) < 1e-12


@pytest.mark.parametrize("n", [(20, 12, 18), (12, 10, 15), (128, 128, 128), (256, 300, 256)])
def test_dealias_band_count_closed_form(n):
    """P keeps exactly (2K0+1)(2K1+1)(K2+1) half-spectrum modes, K_a = (n_a-1)//3,
    and a product of two band modes never aliases back into the band."""
    g = O.Grid(n)
    K = [(m - 1) // 3 for m in n]
    assert int(g.band.sum()) == (2 * K[0] + 1) * (2 * K[1] + 1) * (K[2] + 1)
    for a in range(3):
        assert 2 * K[a] - n[a] < -K[a]  # the alias of the largest sum lies outside the band


def _dense_operator(g, apply):
    m = 3 * int(np.prod(g.n))
    A = np.empty((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        A[:, j] = apply(e.reshape((3,) + g.n)).ravel()
    return A


def _krylov_galerkin_iterates(H, K, b, kmax):
    """The PCG iterates characterised without the CG recurrence: x_k is the
    Galerkin (H-orthogonal) projection of the solution of H x = b onto the
    preconditioned Krylov space span{K b, (K H) K b, ..., (K H)^(k-1) K b}."""
    xs, Q = [], np.zeros((b.size, 0))
    v = K @ b
    for _ in range(kmax):
        for _ in range(2):
            v = v - Q @ (Q.T @ v)
        Q = np.hstack([Q, (v / np.linalg.norm(v))[:, None]])
        xs.append(Q @ np.linalg.solve(Q.T @ H @ Q, Q.T @ b))
        v = K @ (H @ Q[:, -1])
    return xs


def test_pcg_stopping_test_in_V_and_L2():
    """PCG with preconditioner K stops at the first iteration whose residual,
    measured in the norm of the chosen space (V: sqrt(<r, K r>); L2: ||r||),
    is at most rtol times the initial one (reading C9 of the V / L2 variants
    of Sec. 3).  The expected iteration and iterate come from the Galerkin
    characterisation of PCG on the dense 4^3 Gauss-Newton Hessian; alpha = 1
    makes K far from the identity, so the two norms stop at different
    iterations for every rtol used here."""
    n = (4, 4, 4)
    g = O.Grid(n, alpha=1.0)
    p = O.Params(alpha=1.0, nt=4, weight=1e-2)
    r = synth.rng_for(70)
    I0 = synth.spectral_gaussian_smooth(r.standard_normal(n), 0.6)
    I1 = synth.spectral_gaussian_smooth(r.standard_normal(n), 0.6)
    v0 = 0.3 * synth.spectral_gaussian_smooth(r.standard_normal(n), 0.6)[None] * np.array(
        [1.0, -0.5, 0.8]).reshape(3, 1, 1, 1)
    gl2, _, _, _, tr = O.gradient(g, p, v0, I0, I1)
    H = _dense_hessian(g, p, tr)
    K = _dense_operator(g, g.K)
    b = -gl2.ravel()
    xs = _krylov_galerkin_iterates(H, K, b, 8)
    res = {"V": [math.sqrt(b @ K @ b)], "L2": [float(np.linalg.norm(b))]}
    for x in xs:
        rk = b - H @ x
        res["V"].append(math.sqrt(rk @ K @ rk))
        res["L2"].append(float(np.linalg.norm(rk)))
    for rtol in (0.45, 0.105, 0.04):
        want = {s: next(k for k in range(1, 9) if res[s][k] <= rtol * res[s][0]) for s in res}
        assert want["V"] != want["L2"], (rtol, want)
        for space in ("V", "L2"):
            x, it = O.pcg(g, lambda d: O.hessvec(g, p, tr, d), -gl2, g.K, 20, rtol, space)
            assert it == want[space], (rtol, space, it, want)
            assert rel(x.ravel(), xs[it - 1]) < 1e-9


def test_gauss_newton_armijo_acceptance():
    """Each accepted Gauss-Newton step eps (update v0 <- v0 + eps x with
    H x = -g, Sec. 3 with reading C1) satisfies the Armijo condition
    E(v + eps x) <= E(v) + c1 eps <g, x>, recomputed here from the energy,
    and, when eps < 1, the doubled step does not (halving from eps = 1).
    c1 = 0.45 makes the condition decide: two of the four steps are halved."""
    g = O.Grid((6, 6, 6), alpha=0.05)
    p = O.Params(alpha=0.05, nt=4, weight=1e-3)
    I0, vtrue = synth.blob_pair_inputs(g.n, 95, kmax=2, max_disp_vox=3.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = O.shoot(g, vtrue, p.nt, I0).m1
    c1 = 0.45
    rep = O.register(g, p, I0, I1, gn_maxit=4, pcg_maxit=8, c1=c1)
    assert any(e < 1.0 for e in rep.steps) and any(e == 1.0 for e in rep.steps)
    v = np.zeros((3,) + g.n)
    for it, eps in zip(rep.pcg_iters, rep.steps):
        gl2, E, _, _, tr = O.gradient(g, p, v, I0, I1)
        x, _ = O.pcg(g, lambda d: O.hessvec(g, p, tr, d), -gl2, g.K, it, 0.0, force_iters=it)
        slope = g.dot(gl2, x)
        assert slope < 0.0
        assert O.energy(g, p, v + eps * x, I0, I1)[0] <= E + c1 * eps * slope
        if eps < 1.0:
            assert O.energy(g, p, v + 2 * eps * x, I0, I1)[0] > E + c1 * 2 * eps * slope
        v = v + eps * x
    assert rel(v, rep.v0) < 1e-13


def test_threaded_fft_backend_gives_the_same_operators():
    """The scipy.fft backend with worker threads (used only to time the
    oracle on several cores) computes the same spectral operators as
    numpy.fft, to rounding."""
    g = O.Grid((12, 10, 14), alpha=0.05)
    v = rough(g.n, 80)
    ref = (g.K(v), g.P(v), g.grad(v[0]))
    O.set_fft_workers(4)
    try:
        got = (g.K(v), g.P(v), g.grad(v[0]))
    finally:
        O.set_fft_workers(None)
    for a, b in zip(got, ref):
        assert rel(a, b) < 1e-14
