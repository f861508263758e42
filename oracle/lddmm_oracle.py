"""Plain FP64 CPU oracle of the PDE-EPDiff LDDMM hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  It
shares no code with the CUDA path and imports nothing from the package.

What it computes (Hernandez, "PDE-constrained LDDMM via geodesic shooting
and inexact Gauss-Newton-Krylov optimization using the incremental adjoint
Jacobi equations", arXiv 1807.04638):

* the metric ``L = (Id - alpha Lap)^s`` and ``K = L^-1`` (Sec. 2.1),
* the EPDiff right-hand side ``dv/dt = -K ad*_v L v`` with
  ``ad*_v m = (Dv)^T m + (Dm) v + m div v`` (Sec. 2.2, the EPDiff equation),
* geodesic shooting of ``v0`` and transport of the source image,
  ``m(1) = I0 o (phi_1)^-1`` (Sec. 3, state equation),
* the energy ``E(v0) = w <L v0, v0> + ||m(1) - I1||^2`` (Sec. 3; ``w`` plays
  the role of ``sigma^2``),
* the reduced gradient: ``grad_{v1} E = lambda(1) grad m(1)`` with
  ``lambda(1) = -2 (m(1) - I1)``, carried back to ``t = 0`` by the adjoint
  Jacobi equations (Sec. 2.2 and Sec. 3),
* the Gauss-Newton Hessian-vector product: incremental EPDiff forward, the
  Gauss-Newton source ``delta lambda(1) grad m(1)`` with
  ``delta lambda(1) = -2 delta m(1)``, carried back by the same adjoint sweep
  (Sec. 3, with the paper's Gauss-Newton drops),
* PCG with preconditioner ``K`` on ``H dv0 = -grad E`` and the Gauss-Newton
  update of ``v0`` (Sec. 2.3 and Sec. 3), plus the reporting metrics of
  Sec. 4 (relative MSE, relative gradient sup-norm, Jacobian determinant).

Discretisation choices where the paper is silent (each restated where used):
pseudo-spectral derivatives on a periodic grid with the Nyquist mode of first
derivatives zeroed; Heun time stepping of the shooting and of the augmented
Jacobi system; the backward sweep is the exact discrete transpose of the
forward tangent sweep; semi-Lagrangian transport of the inverse-map
displacement with a Heun backward characteristic; Catmull-Rom (Keys, a=-1/2)
or trilinear periodic interpolation.

Layout: scalar fields ``[n0, n1, n2]``; vector fields ``[3, n0, n1, n2]``;
component ``c`` of a vector field is its displacement / velocity along axis
``c``.  Inner products ``<f, g> = h0 h1 h2 sum_x sum_c f_c g_c``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

AXES = (-3, -2, -1)

# FFT backend: numpy's pocketfft on one thread (default), or scipy.fft with
# worker threads (the same transform, used to time the oracle on several
# host cores).
_FFT_WORKERS = None


def set_fft_workers(workers=None):
    """Route the oracle's transforms through scipy.fft with `workers`
    threads; None restores numpy.fft."""
    global _FFT_WORKERS
    _FFT_WORKERS = workers


# ---------------------------------------------------------------------------
# Grid, symbols and spectral operators (Sec. 2.1: L = (Id - alpha Lap)^s)
# ---------------------------------------------------------------------------

class Grid:
    """Periodic grid with spectral symbols.

    ``kappa_a = (2 pi / l_a) k_a`` with integer ``k_a`` in FFT order.  The
    first-derivative symbol ``i kappa_a`` has its Nyquist entry zeroed (so the
    discrete derivative is real and exactly skew-symmetric); ``|kappa|^2``
    keeps the Nyquist entry.  ``L_hat = (1 + alpha |kappa|^2)^s``.

    ``dealias``: the spectral projector P keeps the modes with
    |k_a| <= floor((n_a - 1) / 3) on every axis (the 2/3 rule), so that a
    product of two band-limited fields is resolved exactly after P.  With
    ``dealias=False`` P is the identity.
    """

    def __init__(self, n, alpha=0.01, s=2, lengths=None, dealias=True):
        self.n = tuple(int(x) for x in n)
        self.lengths = tuple(float(x) for x in lengths) if lengths is not None else (2 * math.pi,) * 3
        self.h = tuple(l / m for l, m in zip(self.lengths, self.n))
        self.alpha = float(alpha)
        self.s = int(s)
        self.cell = self.h[0] * self.h[1] * self.h[2]
        # integer wave numbers in FFT order (rounded: fftfreq * n is not exact)
        k = [np.rint(np.fft.fftfreq(self.n[0]) * self.n[0]),
             np.rint(np.fft.fftfreq(self.n[1]) * self.n[1]),
             np.rint(np.fft.rfftfreq(self.n[2]) * self.n[2])]
        kap = [2 * math.pi / self.lengths[a] * k[a] for a in range(3)]
        dsym = []
        for a in range(3):
            d = kap[a].copy()
            if self.n[a] % 2 == 0:
                d[np.abs(k[a]) == self.n[a] // 2] = 0.0
            dsym.append(d)
        shp = [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]
        self.ik = [1j * dsym[a].reshape(shp[a]) for a in range(3)]
        ksq = sum(kap[a].reshape(shp[a]) ** 2 for a in range(3))
        self.ksq = ksq
        self.Lhat = (1.0 + self.alpha * ksq) ** self.s
        self.Khat = 1.0 / self.Lhat
        self.dealias = bool(dealias)
        cut = [(m - 1) // 3 for m in self.n]
        inb = [np.abs(k[a]) <= cut[a] for a in range(3)]
        self.band = (inb[0].reshape(shp[0]) & inb[1].reshape(shp[1]) & inb[2].reshape(shp[2]))
        if not self.dealias:
            self.band = np.ones_like(self.band)
        self.coords = np.stack(np.meshgrid(*[np.arange(m, dtype=np.float64) for m in self.n],
                                           indexing="ij"))

    # transforms --------------------------------------------------------
    def fwd(self, f):
        if _FFT_WORKERS:
            import scipy.fft
            return scipy.fft.rfftn(f, axes=AXES, workers=_FFT_WORKERS)
        return np.fft.rfftn(f, axes=AXES)

    def inv(self, F):
        if _FFT_WORKERS:
            import scipy.fft
            return scipy.fft.irfftn(F, s=self.n, axes=AXES, workers=_FFT_WORKERS)
        return np.fft.irfftn(F, s=self.n, axes=AXES)

    # operators on real fields -----------------------------------------
    def D(self, f, j):
        """Spectral first derivative along axis j (acts on the last 3 axes)."""
        return self.inv(self.ik[j] * self.fwd(f))

    def grad(self, f):
        F = self.fwd(f)
        return np.stack([self.inv(self.ik[j] * F) for j in range(3)])

    def jac(self, v):
        """J[i, j] = D_j v_i."""
        V = self.fwd(v)
        return np.stack([np.stack([self.inv(self.ik[j] * V[i]) for j in range(3)]) for i in range(3)])

    def div(self, v):
        V = self.fwd(v)
        return self.inv(sum(self.ik[j] * V[j] for j in range(3)))

    def L(self, v):
        return self.inv(self.Lhat * self.fwd(v))

    def K(self, v):
        return self.inv(self.Khat * self.fwd(v))

    def P(self, v):
        """2/3-rule projector (identity when dealiasing is off)."""
        return self.inv(self.band * self.fwd(v)) if self.dealias else np.array(v, dtype=np.float64)

    def dot(self, f, g):
        return float(self.cell * np.sum(np.asarray(f) * np.asarray(g)))


# ---------------------------------------------------------------------------
# ad* and ad (Sec. 2.2, EPDiff equation) and their exact discrete transposes
# ---------------------------------------------------------------------------

def ad_star(g: Grid, v, m):
    """ad*_v m = (Dv)^T m + (Dm) v + m div v  (the bracket in the EPDiff equation).

    [(Dv)^T m]_i = sum_j (D_i v_j) m_j ;  [(Dm) v]_i = sum_j (D_j m_i) v_j.
    """
    Jv = g.jac(v)
    Jm = g.jac(m)
    divv = Jv[0, 0] + Jv[1, 1] + Jv[2, 2]
    out = np.empty_like(v)
    for i in range(3):
        out[i] = (sum(Jv[j, i] * m[j] for j in range(3))
                  + sum(Jm[i, j] * v[j] for j in range(3))
                  + m[i] * divv)
    return out


def ad(g: Grid, v, w):
    """ad_v w = (Dv) w - (Dw) v, the L2-dual of ad*_v (continuum identity
    <ad*_v m, w> = <m, ad_v w>)."""
    Jv = g.jac(v)
    Jw = g.jac(w)
    out = np.empty_like(v)
    for i in range(3):
        out[i] = sum(Jv[i, j] * w[j] - Jw[i, j] * v[j] for j in range(3))
    return out


def ad_star_T_first(g: Grid, m, y):
    """Exact grid transpose of eta -> ad*_eta m, applied to y.

    [.]_j = -sum_i D_i(m_j y_i) + sum_i (D_j m_i) y_i - D_j(m . y).
    """
    Jm = g.jac(m)
    my = sum(m[i] * y[i] for i in range(3))
    gmy = g.grad(my)
    out = np.empty_like(y)
    for j in range(3):
        out[j] = (-g.div(np.stack([m[j] * y[i] for i in range(3)]))
                  + sum(Jm[i, j] * y[i] for i in range(3))
                  - gmy[j])
    return out


def ad_star_T_second(g: Grid, v, y):
    """Exact grid transpose of mu -> ad*_v mu, applied to y.

    [.]_k = sum_i (D_i v_k) y_i - sum_j D_j(v_j y_k) + (div v) y_k.
    """
    Jv = g.jac(v)
    divv = Jv[0, 0] + Jv[1, 1] + Jv[2, 2]
    out = np.empty_like(y)
    for k in range(3):
        out[k] = (sum(Jv[k, i] * y[i] for i in range(3))
                  - g.div(np.stack([v[j] * y[k] for j in range(3)]))
                  + divv * y[k])
    return out


def ad_T(g: Grid, v, y):
    """Exact grid transpose of xi -> ad_v xi, applied to y.

    [.]_k = sum_i (D_k v_i) y_i + sum_j D_j(v_j y_k).
    """
    Jv = g.jac(v)
    out = np.empty_like(y)
    for k in range(3):
        out[k] = (sum(Jv[i, k] * y[i] for i in range(3))
                  + g.div(np.stack([v[j] * y[k] for j in range(3)])))
    return out


# ---------------------------------------------------------------------------
# EPDiff right-hand side and its linearisation (Sec. 2.2; Sec. 3 incremental
# EPDiff equation)
# ---------------------------------------------------------------------------

def epdiff_rhs(g: Grid, v):
    """R(v) = -K P ad*_v (L v)  (P: the dealiasing projector of the products)."""
    return -g.K(g.P(ad_star(g, v, g.L(v))))


def epdiff_rhs_lin(g: Grid, v, eta):
    """R'(v) eta = -K P [ad*_eta (L v) + ad*_v (L eta)]  (incremental EPDiff:
    d/dt dv = -(ad^dagger_dv v + ad^dagger_v dv))."""
    return -g.K(g.P(ad_star(g, eta, g.L(v)) + ad_star(g, v, g.L(eta))))


def epdiff_rhs_lin_T(g: Grid, v, y):
    """Exact grid transpose of eta -> R'(v) eta."""
    PKy = g.P(g.K(y))
    return -(ad_star_T_first(g, g.L(v), PKy) + g.L(ad_star_T_second(g, v, PKy)))


# ---------------------------------------------------------------------------
# Periodic interpolation and semi-Lagrangian map transport (Sec. 3 state
# equation  dm/dt + grad m . v = 0, solved through the inverse map)
# ---------------------------------------------------------------------------

def _catmull_rom_weights(t):
    t2 = t * t
    t3 = t2 * t
    return [0.5 * (-t3 + 2 * t2 - t),
            0.5 * (3 * t3 - 5 * t2 + 2),
            0.5 * (-3 * t3 + 4 * t2 + t),
            0.5 * (t3 - t2)]


def interp(f, p, kind="cubic"):
    """Periodic interpolation of samples ``f`` (last 3 axes) at voxel
    coordinates ``p`` (shape [3, ...]).  ``kind`` = 'cubic' (Catmull-Rom,
    Keys a=-1/2, taps -1..2) or 'linear' (trilinear, taps 0..1)."""
    f = np.asarray(f)
    n = f.shape[-3:]
    base = np.floor(p)
    t = p - base
    base = base.astype(np.int64)
    if kind == "cubic":
        offs = (-1, 0, 1, 2)
        w = [_catmull_rom_weights(t[a]) for a in range(3)]
    elif kind == "linear":
        offs = (0, 1)
        w = [[1.0 - t[a], t[a]] for a in range(3)]
    else:
        raise ValueError(kind)
    lead = f.shape[:-3]
    out = np.zeros(lead + p.shape[1:])
    for a0, o0 in enumerate(offs):
        i0 = np.mod(base[0] + o0, n[0])
        for a1, o1 in enumerate(offs):
            i1 = np.mod(base[1] + o1, n[1])
            w01 = w[0][a0] * w[1][a1]
            for a2, o2 in enumerate(offs):
                i2 = np.mod(base[2] + o2, n[2])
                out += (w01 * w[2][a2]) * f[..., i0, i1, i2]
    return out


def sl_map_step(g: Grid, u_k, v_k, v_k1, dt, kind="cubic"):
    """One semi-Lagrangian step of the inverse-map displacement u
    (psi_t = x + u_t = phi_t^-1), Heun backward characteristic:

      Xt = x - dt v_{k+1}(x);   X = x - dt/2 (v_{k+1}(x) + v_k(Xt));
      u_{k+1}(x) = (X - x) + u_k(X).
    """
    h = np.array(g.h).reshape(3, 1, 1, 1)
    x = g.coords
    p1 = x - dt * v_k1 / h
    vt = interp(v_k, p1, kind)
    disp = -0.5 * dt * (v_k1 + vt)
    return disp + interp(u_k, x + disp / h, kind)


def warp(g: Grid, img, u, kind="cubic"):
    """m(x) = I(x + u(x))."""
    h = np.array(g.h).reshape(3, 1, 1, 1)
    return interp(img, g.coords + u / h, kind)


# ---------------------------------------------------------------------------
# Geodesic shooting (Heun) with map transport
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Trajectory:
    nt: int
    v: List[np.ndarray]        # v_k, k = 0..nt
    vstar: List[np.ndarray]    # Heun predictors v*_k, k = 0..nt-1
    u: np.ndarray              # inverse-map displacement at t = 1
    kinetic: List[float]       # <L v_k, v_k>, k = 0..nt
    m1: Optional[np.ndarray] = None
    grad_m1: Optional[np.ndarray] = None


def shoot(g: Grid, v0, nt, I0=None, kind="cubic", transport=True):
    """Forward geodesic shooting of P v0 by Heun steps of the EPDiff
    equation, with SL transport of the inverse map and the final warp
    m(1) = I0(x+u).  ``transport=False`` keeps u = 0 and m(1) = I0 (the
    EPDiff states alone; used to time the sweeps without the transport)."""
    dt = 1.0 / nt
    v = [g.P(v0)]
    vstar = []
    u = np.zeros_like(v[0])
    for k in range(nt):
        r1 = epdiff_rhs(g, v[k])
        vs = v[k] + dt * r1
        r2 = epdiff_rhs(g, vs)
        v.append(v[k] + 0.5 * dt * (r1 + r2))
        vstar.append(vs)
        if transport:
            u = sl_map_step(g, u, v[k], v[k + 1], dt, kind)
    kin = [g.dot(g.L(vk), vk) for vk in v]
    tr = Trajectory(nt=nt, v=v, vstar=vstar, u=u, kinetic=kin)
    if I0 is not None:
        tr.m1 = warp(g, I0, u, kind) if transport else np.array(I0, dtype=np.float64)
        tr.grad_m1 = g.grad(tr.m1)
    return tr


# ---------------------------------------------------------------------------
# Jacobi sweeps: forward tangent T and its exact transpose T^T
# (Sec. 3: incremental EPDiff forward; adjoint / incremental adjoint Jacobi
# field equations backward)
# ---------------------------------------------------------------------------

def jacobi_A(g: Grid, v, eta, xi):
    """A_v(eta, xi) = (R'(v) eta, eta + P ad_v xi); the Jacobi field equation
    xi' = eta + ad_v xi is the right-trivialised variation of the flow."""
    return epdiff_rhs_lin(g, v, eta), eta + g.P(ad(g, v, xi))


def jacobi_A_T(g: Grid, v, yeta, yxi):
    """Exact grid transpose of jacobi_A."""
    return epdiff_rhs_lin_T(g, v, yeta) + yxi, ad_T(g, v, g.P(yxi))


def tangent(g: Grid, tr: Trajectory, delta):
    """T: delta v0 -> (eta_nt, xi_nt), Heun on the augmented system reusing the
    stored states (v_k for stage 1, v*_k for stage 2), from (P delta, 0)."""
    dt = 1.0 / tr.nt
    eta = g.P(delta)
    xi = np.zeros_like(eta)
    for k in range(tr.nt):
        be, bx = jacobi_A(g, tr.v[k], eta, xi)
        es, xs = eta + dt * be, xi + dt * bx
        ce, cx = jacobi_A(g, tr.vstar[k], es, xs)
        eta = eta + 0.5 * dt * (be + ce)
        xi = xi + 0.5 * dt * (bx + cx)
    return eta, xi


def adjoint(g: Grid, tr: Trajectory, b_xi, b_eta=None):
    """T^T: exact transpose of ``tangent``.  Given the cotangent (b_eta, b_xi)
    on (eta_nt, xi_nt), returns the cotangent on delta v0.

    Per step (reverse order), with z' = z + dt/2 A z + dt/2 A*(z + dt A z):
      a = A*^T zbar;  zbar <- zbar + dt/2 a + A^T (dt/2 zbar + dt^2/2 a).
    """
    dt = 1.0 / tr.nt
    yx = np.array(b_xi, dtype=np.float64)
    ye = np.zeros_like(yx) if b_eta is None else np.array(b_eta, dtype=np.float64)
    for k in reversed(range(tr.nt)):
        ae, ax = jacobi_A_T(g, tr.vstar[k], ye, yx)
        te, tx = jacobi_A_T(g, tr.v[k], 0.5 * dt * ye + 0.5 * dt * dt * ae,
                            0.5 * dt * yx + 0.5 * dt * dt * ax)
        ye = ye + 0.5 * dt * ae + te
        yx = yx + 0.5 * dt * ax + tx
    return g.P(ye)


# ---------------------------------------------------------------------------
# Energy, gradient, Gauss-Newton Hessian-vector product (Sec. 3)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    alpha: float = 0.01
    s: int = 2
    weight: float = 1e-3       # w = sigma^2: E = w <L v0, v0> + ||m1 - I1||^2
    nt: int = 10
    interp: str = "cubic"
    space: str = "V"           # 'V' or 'L2'


def energy(g: Grid, p: Params, v0, I0, I1, tr=None):
    """E(v0) = w <L v0, v0> + ||m(1) - I1||^2 with m(1) shot from P v0;
    returns (E, data, reg, tr)."""
    if tr is None:
        tr = shoot(g, v0, p.nt, I0, p.interp)
    r = tr.m1 - I1
    data = g.dot(r, r)
    reg = p.weight * g.dot(g.L(v0), v0)
    return data + reg, data, reg, tr


def gradient(g: Grid, p: Params, v0, I0, I1):
    """Reduced L2 gradient  g = 2 w L v0 + T^T b,  b = lambda(1) grad m(1),
    lambda(1) = -2 (m(1) - I1).  Returns (g_L2, E, data, reg, tr)."""
    E, data, reg, tr = energy(g, p, v0, I0, I1)
    b = -2.0 * (tr.m1 - I1)[None] * tr.grad_m1
    gl2 = 2.0 * p.weight * g.L(v0) + adjoint(g, tr, b)
    return gl2, E, data, reg, tr


def hessvec(g: Grid, p: Params, tr: Trajectory, dv0):
    """Gauss-Newton L2 Hessian-vector product at the trajectory tr:

      H dv0 = 2 w L dv0 + T^T c,  with  delta m(1) = -grad m(1) . xi(1),
      delta lambda(1) = -2 delta m(1)  and the Gauss-Newton source
      c = delta lambda(1) grad m(1) = 2 (grad m(1) . xi(1)) grad m(1)
      (the lambda(1) grad delta m(1) term is dropped).
    """
    _, xi = tangent(g, tr, dv0)
    dm1 = -np.sum(tr.grad_m1 * xi, axis=0)
    c = -2.0 * dm1[None] * tr.grad_m1
    return 2.0 * p.weight * g.L(dv0) + adjoint(g, tr, c)


def to_space(g: Grid, p: Params, f):
    """Metric of the returned gradient / Hessian product: V -> K f, L2 -> f."""
    return g.K(f) if p.space == "V" else f


# ---------------------------------------------------------------------------
# PCG and the Gauss-Newton-Krylov loop (Sec. 2.3 / Sec. 3)
# ---------------------------------------------------------------------------

def pcg(g: Grid, hmul: Callable, rhs, precond: Callable, maxit, rtol, space="V",
        force_iters=None):
    """PCG on H x = rhs with preconditioner K, x0 = 0.

    Stopping norm relative to iteration 0: V -> sqrt(<r, K r>), L2 -> ||r||.
    Stops early when <p, H p> <= 0.  ``force_iters`` replays a given iteration
    count instead of the stopping test.  Returns (x, iterations).
    """
    x = np.zeros_like(rhs)
    r = np.array(rhs, dtype=np.float64)
    z = precond(r)
    pdir = z.copy()
    rz = g.dot(r, z)
    norm0 = math.sqrt(max(rz, 0.0)) if space == "V" else math.sqrt(g.dot(r, r))
    it = 0
    limit = maxit if force_iters is None else force_iters
    while it < limit:
        q = hmul(pdir)
        pq = g.dot(pdir, q)
        if pq <= 0.0:
            break
        alpha = rz / pq
        x = x + alpha * pdir
        r = r - alpha * q
        z = precond(r)
        rz_new = g.dot(r, z)
        it += 1
        res = math.sqrt(max(rz_new, 0.0)) if space == "V" else math.sqrt(g.dot(r, r))
        if force_iters is None and res <= rtol * norm0:
            break
        beta = rz_new / rz
        pdir = z + beta * pdir
        rz = rz_new
    return x, it


@dataclasses.dataclass
class GNReport:
    energies: List[float]
    pcg_iters: List[int]
    steps: List[float]
    gnorm_rel: float
    mse_rel: float
    jac_min: float
    jac_max: float
    v0: np.ndarray


def jacobian_det(g: Grid, u):
    """det(I + D u) of the inverse map psi = x + u (spectral derivatives)."""
    J = g.jac(u)
    a = J + np.eye(3).reshape(3, 3, 1, 1, 1)
    return (a[0, 0] * (a[1, 1] * a[2, 2] - a[1, 2] * a[2, 1])
            - a[0, 1] * (a[1, 0] * a[2, 2] - a[1, 2] * a[2, 0])
            + a[0, 2] * (a[1, 0] * a[2, 1] - a[1, 1] * a[2, 0]))


def register(g: Grid, p: Params, I0, I1, v0=None, gn_maxit=5, pcg_maxit=10, pcg_rtol=0.1,
             c1=1e-4, ls_maxit=10, replay=None, exact_gradient=False):
    """Inexact Gauss-Newton-Krylov registration in the space of initial
    velocities.  Update v0 <- v0 + eps dv0 with H dv0 = -g (the descent sign;
    the paper writes the update with the opposite sign convention on dv0),
    Armijo backtracking from eps = 1 with halving.

    ``replay`` = list of (pcg_iterations, eps) per GN iteration forces the
    decisions (used to compare trajectories computed at another precision).
    ``exact_gradient`` uses the gradient of the discrete energy
    (``gradient_exact``) in place of the Jacobi-field gradient; the
    Gauss-Newton Hessian is the same.
    """
    v = np.zeros((3,) + g.n) if v0 is None else np.array(v0, dtype=np.float64)
    energies, iters, steps = [], [], []
    g0max = None
    gmax = None
    for n_it in range(gn_maxit):
        gl2, E, _, _, tr = gradient(g, p, v, I0, I1)
        if exact_gradient:
            gl2 = gradient_exact(g, p, v, I0, I1)[0]
        gsp = to_space(g, p, gl2)
        gmax = float(np.abs(gsp).max())
        if g0max is None:
            g0max = gmax
        energies.append(E)
        forced = replay[n_it] if replay is not None else None
        x, it = pcg(g, lambda d: hessvec(g, p, tr, d), -gl2, g.K, pcg_maxit, pcg_rtol,
                    p.space, force_iters=None if forced is None else forced[0])
        iters.append(it)
        slope = g.dot(gl2, x)
        if forced is not None:
            eps = forced[1]
        else:
            eps = 1.0
            accepted = False
            for _ in range(ls_maxit):
                Et = energy(g, p, v + eps * x, I0, I1)[0]
                if Et <= E + c1 * eps * slope:
                    accepted = True
                    break
                eps *= 0.5
            if not accepted:
                eps = 0.0
        steps.append(eps)
        if eps == 0.0:
            break
        v = v + eps * x
    Ef, _, _, trf = energy(g, p, v, I0, I1)
    energies.append(Ef)
    gl2f = gradient_exact(g, p, v, I0, I1)[0] if exact_gradient else gradient(g, p, v, I0, I1)[0]
    gnorm_rel = float(np.abs(to_space(g, p, gl2f)).max() / g0max) if g0max else 0.0
    mse = g.dot(trf.m1 - I1, trf.m1 - I1) / g.dot(I0 - I1, I0 - I1)
    J = jacobian_det(g, trf.u)
    return GNReport(energies=energies, pcg_iters=iters, steps=steps, gnorm_rel=gnorm_rel,
                    mse_rel=float(mse), jac_min=float(J.min()), jac_max=float(J.max()), v0=v)


def register_gd(g: Grid, p: Params, I0, I1, v0=None, maxit=50, c1=1e-4, ls_maxit=10, replay=None):
    """Gradient descent in V on E(v0), the optimisation of Sec. 2.2:
    v0 <- v0 - eps grad_V E with grad_V E = K g_L2 (the V-Riesz representer of
    the reduced gradient).  The paper gives no step rule; this reading uses
    Armijo backtracking with halving, starting in the first iteration at the
    step that moves max |K g_L2| by one voxel (min_a h_a) and afterwards at
    twice the last accepted step.

    ``replay`` = list of eps per iteration forces the steps.
    """
    v = np.zeros((3,) + g.n) if v0 is None else np.array(v0, dtype=np.float64)
    energies, iters, steps = [], [], []
    g0max = None
    eps_prev = None
    hmin = min(g.h)
    for n_it in range(maxit):
        gl2, E, _, _, _ = gradient(g, p, v, I0, I1)
        energies.append(E)
        gV = g.K(gl2)
        if g0max is None:
            g0max = float(np.abs(gV if p.space == "V" else gl2).max())
        x = -gV
        slope = g.dot(gl2, x)
        iters.append(0)
        if replay is not None:
            eps = replay[n_it]
        else:
            kgmax = float(np.abs(gV).max())
            eps = (hmin / kgmax if kgmax > 0 else 1.0) if eps_prev is None else 2.0 * eps_prev
            accepted = False
            for _ in range(ls_maxit):
                Et = energy(g, p, v + eps * x, I0, I1)[0]
                if Et <= E + c1 * eps * slope:
                    accepted = True
                    break
                eps *= 0.5
            if not accepted:
                eps = 0.0
        steps.append(eps)
        if eps == 0.0:
            break
        eps_prev = eps
        v = v + eps * x
    Ef, _, _, trf = energy(g, p, v, I0, I1)
    energies.append(Ef)
    gl2f = gradient(g, p, v, I0, I1)[0]
    gnorm_rel = float(np.abs(to_space(g, p, gl2f)).max() / g0max) if g0max else 0.0
    mse = g.dot(trf.m1 - I1, trf.m1 - I1) / g.dot(I0 - I1, I0 - I1)
    J = jacobian_det(g, trf.u)
    return GNReport(energies=energies, pcg_iters=iters, steps=steps, gnorm_rel=gnorm_rel,
                    mse_rel=float(mse), jac_min=float(J.min()), jac_max=float(J.max()), v0=v)


# ---------------------------------------------------------------------------
# Cross-check of the linearised final image (Sec. 3, incremental state
# equation): the literal route, for comparison with delta m(1) = -grad m(1) .
# xi(1) used by the sweeps.  Not part of the path.
# ---------------------------------------------------------------------------

def tangent_path(g: Grid, tr: Trajectory, delta):
    """The tangent sweep of ``tangent``, returning eta_k for k = 0..nt and
    xi_nt (the same Heun steps)."""
    dt = 1.0 / tr.nt
    eta = g.P(delta)
    xi = np.zeros_like(eta)
    etas = [eta]
    for k in range(tr.nt):
        be, bx = jacobi_A(g, tr.v[k], eta, xi)
        es, xs = eta + dt * be, xi + dt * bx
        ce, cx = jacobi_A(g, tr.vstar[k], es, xs)
        eta = eta + 0.5 * dt * (be + ce)
        xi = xi + 0.5 * dt * (bx + cx)
        etas.append(eta)
    return etas, xi


def incremental_state_literal(g: Grid, tr: Trajectory, I0, etas, kind="cubic"):
    """delta m(1) from the incremental state equation of Sec. 3,
      d/dt delta m + grad(delta m) . v + grad m . delta v = 0,  delta m(0) = 0,
    with delta v = eta (the incremental EPDiff solution) and m_t = I0 o psi_t.
    Along the characteristics of the map step (departure point X of
    ``sl_map_step``) the equation reads d/dt delta m = -grad m . eta, which is
    integrated by the trapezoidal rule:
      dm_{k+1}(x) = dm_k(X) - dt/2 [(grad m_{k+1} . eta_{k+1})(x)
                                    + (grad m_k . eta_k)(X)]."""
    dt = 1.0 / tr.nt
    h = np.array(g.h).reshape(3, 1, 1, 1)
    x = g.coords
    u = np.zeros((3,) + g.n)
    src = np.sum(g.grad(I0) * etas[0], axis=0)
    dm = np.zeros(g.n)
    for k in range(tr.nt):
        v0_, v1_ = tr.v[k], tr.v[k + 1]
        u = sl_map_step(g, u, v0_, v1_, dt, kind)
        m1_ = warp(g, I0, u, kind)
        src1 = np.sum(g.grad(m1_) * etas[k + 1], axis=0)
        vt = interp(v0_, x - dt * v1_ / h, kind)
        X = x + (-0.5 * dt * (v1_ + vt)) / h
        dm = interp(dm, X, kind) - 0.5 * dt * (src1 + interp(src, X, kind))
        src = src1
    return dm


# ---------------------------------------------------------------------------
# Exact discrete adjoint of the semi-Lagrangian transport (discretise-then-
# optimise gradient).  The energy of the discrete method depends on v0 through
# the stage-1 velocities v_k of the Heun EPDiff steps, which the map steps
# (sl_map_step) and the final warp read by interpolation.  Transposing those
# interpolations (a scatter) and their coordinate derivatives gives dE/dv_k
# exactly; the adjoint of the incremental EPDiff (the eta block of the
# adjoint Jacobi sweep) carries these cotangents back to v0.  The result is
# the gradient of the discrete energy itself, which finite differences
# reproduce to rounding, unlike the Jacobi-field gradient of Sec. 3.
# ---------------------------------------------------------------------------

def _catmull_rom_dweights(t):
    """d/dt of the Catmull-Rom weights."""
    t2 = t * t
    return [0.5 * (-3 * t2 + 4 * t - 1),
            0.5 * (9 * t2 - 10 * t),
            0.5 * (-9 * t2 + 8 * t + 1),
            0.5 * (3 * t2 - 2 * t)]


def _taps(p, kind):
    base = np.floor(p)
    t = p - base
    base = base.astype(np.int64)
    if kind == "cubic":
        offs = (-1, 0, 1, 2)
        w = [_catmull_rom_weights(t[a]) for a in range(3)]
        dw = [_catmull_rom_dweights(t[a]) for a in range(3)]
    elif kind == "linear":
        offs = (0, 1)
        w = [[1.0 - t[a], t[a]] for a in range(3)]
        dw = [[-np.ones_like(t[a]), np.ones_like(t[a])] for a in range(3)]
    else:
        raise ValueError(kind)
    return base, offs, w, dw


def interp_grad(f, p, kind="cubic"):
    """Derivative of ``interp(f, p)`` with respect to the voxel coordinates:
    shape [3] + f's leading axes + points (component a = d/dp_a)."""
    f = np.asarray(f)
    n = f.shape[-3:]
    base, offs, w, dw = _taps(p, kind)
    lead = f.shape[:-3]
    out = np.zeros((3,) + lead + p.shape[1:])
    for a0, o0 in enumerate(offs):
        i0 = np.mod(base[0] + o0, n[0])
        for a1, o1 in enumerate(offs):
            i1 = np.mod(base[1] + o1, n[1])
            for a2, o2 in enumerate(offs):
                i2 = np.mod(base[2] + o2, n[2])
                val = f[..., i0, i1, i2]
                out[0] += (dw[0][a0] * w[1][a1] * w[2][a2]) * val
                out[1] += (w[0][a0] * dw[1][a1] * w[2][a2]) * val
                out[2] += (w[0][a0] * w[1][a1] * dw[2][a2]) * val
    return out


def interp_T(vals, p, n, kind="cubic"):
    """Transpose of ``interp(., p)`` with respect to the samples: scatter
    ``vals`` (leading axes + points) onto the grid n with the same weights."""
    vals = np.asarray(vals)
    base, offs, w, _ = _taps(p, kind)
    lead = vals.shape[:vals.ndim - (p.ndim - 1)]
    out = np.zeros(lead + tuple(n))
    for a0, o0 in enumerate(offs):
        i0 = np.mod(base[0] + o0, n[0])
        for a1, o1 in enumerate(offs):
            i1 = np.mod(base[1] + o1, n[1])
            for a2, o2 in enumerate(offs):
                i2 = np.mod(base[2] + o2, n[2])
                wt = w[0][a0] * w[1][a1] * w[2][a2]
                for li in np.ndindex(*lead):
                    np.add.at(out[li], (i0, i1, i2), wt * vals[li])
    return out


def adjoint_eta_sources(g: Grid, tr: Trajectory, srcs):
    """Transpose of eta_0 = P delta -> (eta_0, ..., eta_nt) of ``tangent``:
    given cotangents srcs[k] on eta_k, returns the cotangent on delta.  The
    xi block of the sweep stays zero (eta does not depend on xi)."""
    dt = 1.0 / tr.nt
    ye = np.array(srcs[tr.nt], dtype=np.float64)
    yx = np.zeros_like(ye)
    for k in reversed(range(tr.nt)):
        ae, ax = jacobi_A_T(g, tr.vstar[k], ye, yx)
        te, tx = jacobi_A_T(g, tr.v[k], 0.5 * dt * ye + 0.5 * dt * dt * ae,
                            0.5 * dt * yx + 0.5 * dt * dt * ax)
        ye = ye + 0.5 * dt * ae + te + srcs[k]
        yx = yx + 0.5 * dt * ax + tx
    return g.P(ye)


def gradient_exact(g: Grid, p: Params, v0, I0, I1):
    """Gradient of the discrete energy E(v0) (shoot, sl_map_step, warp as
    implemented), through the exact transposes of the map steps and of the
    final warp.  Returns (g_L2, E)."""
    kind = p.interp
    dt = 1.0 / p.nt
    h = np.array(g.h).reshape(3, 1, 1, 1)
    x = g.coords
    E, _, _, tr = energy(g, p, v0, I0, I1)
    us = [np.zeros((3,) + g.n)]
    for k in range(p.nt):
        us.append(sl_map_step(g, us[k], tr.v[k], tr.v[k + 1], dt, kind))
    # final warp m1 = I0(x + u_nt / h): dE/du_nt = 2 (m1 - I1) dI0/dp / h
    gI = interp_grad(I0, x + us[p.nt] / h, kind)
    ub = 2.0 * (tr.m1 - I1)[None] * gI / h
    vb = [np.zeros((3,) + g.n) for _ in range(p.nt + 1)]
    for k in reversed(range(p.nt)):
        vk, vk1 = tr.v[k], tr.v[k + 1]
        p1 = x - dt * vk1 / h
        vt = interp(vk, p1, kind)
        disp = -0.5 * dt * (vk1 + vt)
        X = x + disp / h
        # u_{k+1} = disp + interp(u_k, X)
        Gu = interp_grad(us[k], X, kind)               # [b][a]: d u_k,a / d p_b
        dispb = ub + np.einsum("bax,ax->bx", Gu.reshape(3, 3, -1), ub.reshape(3, -1)).reshape(ub.shape) / h
        ubk = interp_T(ub, X, g.n, kind)
        # disp = -dt/2 (v_{k+1} + interp(v_k, p1)),  p1 = x - dt v_{k+1} / h
        vtb = -0.5 * dt * dispb
        vb[k + 1] += -0.5 * dt * dispb
        vb[k] += interp_T(vtb, p1, g.n, kind)
        Gv = interp_grad(vk, p1, kind)
        p1b = np.einsum("bax,ax->bx", Gv.reshape(3, 3, -1), vtb.reshape(3, -1)).reshape(ub.shape)
        vb[k + 1] += -dt * p1b / h
        ub = ubk
    gl2 = 2.0 * p.weight * g.L(v0) + adjoint_eta_sources(g, tr, vb)
    return gl2, E
