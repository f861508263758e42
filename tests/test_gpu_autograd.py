"""Differentiation form: torch.autograd through lddmm_shoot, backward = the
adjoint Jacobi sweep (lddmm_shoot_vjp).

* the backward equals the FP64 oracle's gradient of the same loss
  (P T^T(-G grad m1), G = dloss/dm1) member by member: FP32 within 1e-5,
  FP64 within 1e-10;
* it agrees with central finite differences of the loss (h = 1e-4, random
  band-limited directions, FD through the FP64 shoot) up to the Jacobi-field
  linearisation gap of the semi-Lagrangian warp;
* the batch of eight 96^3 blob-phantom pairs (the differentiation workload)
  runs forward and backward; every member matches the oracle's stored
  gradient, and the backward's gap to the oracle's central differences
  equals the oracle gradient's own gap.
"""
import numpy as np
import pytest

from oracle import lddmm_oracle as O
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


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def batch_inputs(n, seeds, kmax, disp, nt, alpha):
    g = O.Grid(n, alpha=alpha)
    I0s, I1s, v0s = [], [], []
    for s in seeds:
        I0, vt = synth.blob_pair_inputs(n, s, kmax=kmax, max_disp_vox=disp)
        I0 = synth.spectral_gaussian_smooth(I0, 1.0)
        I1s.append(O.shoot(g, vt, nt, I0).m1)
        I0s.append(I0)
        v0s.append(0.6 * vt)
    return g, np.stack(I0s), np.stack(I1s), np.stack(v0s)


def oracle_grad(g, nt, v0, I0, I1):
    tr = O.shoot(g, v0, nt, I0)
    G = 2.0 * (tr.m1 - I1)
    return O.adjoint(g, tr, -G[None] * tr.grad_m1), tr.m1


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_backward_matches_oracle(pkg, prec):
    from paper_1807_04638_gb300.autograd import Shooter, shoot
    n, nt, alpha = (24, 20, 18), 6, 0.01
    g, I0, I1, v0 = batch_inputs(n, [3, 4, 5], 2, 1.5, nt, alpha)
    cd = pkg.LDDMM_F32 if prec == "f32" else pkg.LDDMM_F64
    dt = torch.float32 if prec == "f32" else torch.float64
    sh = Shooter(n, 3, pkg.default_params(alpha=alpha, nt=nt, compute_dtype=cd, state_dtype=cd))
    try:
        v = torch.tensor(v0, dtype=dt, device="cuda", requires_grad=True)
        I0t = torch.tensor(I0, dtype=dt, device="cuda")
        I1t = torch.tensor(I1, dtype=dt, device="cuda")
        m1 = shoot(v, I0t, sh)
        loss = ((m1 - I1t) ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        got = v.grad.double().cpu().numpy()
    finally:
        sh.close()
    tol = 1e-5 if prec == "f32" else 1e-10
    for b in range(3):
        want, m1o = oracle_grad(g, nt, v0[b], I0[b], I1[b])
        assert rel(m1.detach().double().cpu().numpy()[b] - I1[b], m1o - I1[b]) < (1e-4 if prec == "f32" else 1e-10)
        assert rel(got[b], want) < tol, (b, rel(got[b], want))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_checkpointed_backward_equals_stored_states(pkg, prec):
    """When the memory budget asks for it the Shooter checkpoints the forward
    states (every 2 steps) and recomputes them in the backward: the loss
    and the gradient are the same as with every state stored."""
    from paper_1807_04638_gb300.autograd import Shooter, shoot
    n, nt, alpha = (32, 32, 32), 6, 0.01
    g, I0, I1, v0 = batch_inputs(n, [21, 22], 2, 1.5, nt, alpha)
    cd = pkg.LDDMM_F32 if prec == "f32" else pkg.LDDMM_F64
    dt = torch.float32 if prec == "f32" else torch.float64
    prm = pkg.default_params(alpha=alpha, nt=nt, compute_dtype=cd, state_dtype=cd)
    full = pkg.workspace_bytes(n, prm)
    out = []
    for budget in (None, 2 * full - 1):
        sh = Shooter(n, 2, prm, max_bytes=budget)
        try:
            assert sh.params.checkpoint_every == (1 if budget is None else 2)
            v = torch.tensor(v0, dtype=dt, device="cuda", requires_grad=True)
            loss = ((shoot(v, torch.tensor(I0, dtype=dt, device="cuda"), sh)
                     - torch.tensor(I1, dtype=dt, device="cuda")) ** 2).sum()
            loss.backward()
            torch.cuda.synchronize()
            out.append((float(loss.detach()), v.grad.double().cpu().numpy()))
        finally:
            sh.close()
    assert out[0][0] == out[1][0]
    assert rel(out[1][1], out[0][1]) < 1e-12


def test_backward_vs_finite_differences(pkg):
    from paper_1807_04638_gb300.autograd import Shooter, shoot
    n, nt, alpha = (24, 24, 24), 8, 0.01
    g, I0, I1, v0 = batch_inputs(n, [7], 2, 2.0, nt, alpha)
    prm32 = pkg.default_params(alpha=alpha, nt=nt, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    sh = Shooter(n, 1, prm32)
    try:
        v = torch.tensor(v0, dtype=torch.float32, device="cuda", requires_grad=True)
        I0t = torch.tensor(I0, dtype=torch.float32, device="cuda")
        I1t = torch.tensor(I1, dtype=torch.float32, device="cuda")
        loss = ((shoot(v, I0t, sh) - I1t) ** 2).sum()
        loss.backward()
        grad = v.grad.double().cpu().numpy()[0]
    finally:
        sh.close()
    # central differences of the same loss through the FP64 shoot
    with pkg.Handle(n, pkg.default_params(alpha=alpha, nt=nt)) as h:
        I0d = torch.tensor(I0[0], dtype=torch.float64, device="cuda")
        m1 = h.new_img()

        def L(vv):
            h.lddmm_shoot(torch.tensor(vv, dtype=torch.float64, device="cuda"), I0d, m1)
            h.lddmm_synchronize()
            return float(((m1.cpu().numpy() - I1[0]) ** 2).sum())

        r = synth.rng_for(70)
        worst = 0.0
        for _ in range(16):
            d = synth.band_limited_field(n, r, 2.0, 3) * g.h[0]
            eps = 1e-4
            fd = (L(v0[0] + eps * d) - L(v0[0] - eps * d)) / (2 * eps)
            gd = float(np.sum(grad * d))
            worst = max(worst, abs(gd - fd) / (np.linalg.norm(grad) * np.linalg.norm(d)))
    assert worst < 1e-2, worst


def test_batch_of_eight_96_vs_oracle_and_oracle_finite_differences(pkg):
    """The differentiation workload in full: eight independent 96^3 blob
    pairs (nt = 10, FP32 form) forward and backward through the
    autograd.Function, every member against the FP64 oracle's gradient of
    ||m1 - I1||^2 (stored by tests/golden/make_golden.py): values at 2048
    points, the norm, and the projections on 16 band-limited directions,
    each within 1e-5; and, for four members, the gap between the backward
    and the oracle's central differences (h = 1e-4) in those directions
    equals the oracle gradient's own gap within 10% (the Jacobi-field
    linearisation gap of the semi-Lagrangian warp, Sec. 3)."""
    import importlib.util
    import json
    import os
    from paper_1807_04638_gb300.autograd import Shooter, shoot
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(here, "golden", "config4_96cubed.json")) as f:
        ref = json.load(f)
    n, nt, alpha = mg.C4_N, mg.C4_NT, mg.C4_ALPHA
    B = len(mg.C4_SEEDS)
    idx = mg.config4_sample_idx()
    members = [mg.config4_member(b) for b in range(B)]
    I0 = np.stack([m[0] for m in members])
    v0 = np.stack([m[2] for m in members])
    # targets: the FP64 library shoot of each true velocity, checked against
    # the oracle's stored samples and norm first
    I1 = np.empty_like(I0)
    f64 = torch.float64
    with pkg.Handle(n, pkg.default_params(alpha=alpha, nt=nt)) as h64:
        m1 = h64.new_img()
        for b, (I0b, vt, _) in enumerate(members):
            h64.lddmm_shoot(torch.tensor(vt, dtype=f64, device="cuda"), torch.tensor(I0b, dtype=f64, device="cuda"),
                            m1)
            I1[b] = m1.cpu().numpy()
            r = ref["members"][b]
            assert rel(I1[b].ravel()[idx % I1[b].size], r["m1_true"]) < 1e-9
            assert abs(np.linalg.norm(I1[b]) - r["m1_true_l2"]) < 1e-9 * r["m1_true_l2"]
    sh = Shooter(n, B, pkg.default_params(alpha=alpha, nt=nt, compute_dtype=pkg.LDDMM_F32,
                                          state_dtype=pkg.LDDMM_F32))
    try:
        v = torch.tensor(v0, dtype=torch.float32, device="cuda", requires_grad=True)
        I0t = torch.tensor(I0, dtype=torch.float32, device="cuda")
        I1t = torch.tensor(I1, dtype=torch.float32, device="cuda")
        per = ((shoot(v, I0t, sh) - I1t) ** 2).sum(dim=(1, 2, 3))
        per.sum().backward()
        torch.cuda.synchronize()
        grad = v.grad.double().cpu().numpy()
        losses = per.detach().double().cpu().numpy()
    finally:
        sh.close()
    assert np.isfinite(grad).all()
    for b in range(B):
        r = ref["members"][b]
        g = grad[b]
        gn = np.linalg.norm(g)
        assert abs(losses[b] - r["loss"]) < 1e-4 * r["loss"], b
        assert rel(g.ravel()[idx], r["grad"]) < 1e-5, (b, rel(g.ravel()[idx], r["grad"]))
        assert abs(gn - r["grad_l2"]) < 1e-5 * r["grad_l2"], b
        dirs = mg.config4_directions(b)
        for i, d in enumerate(dirs):
            dn = np.linalg.norm(d)
            gd = float(np.sum(g * d))
            assert abs(gd - r["grad_dot_dir"][i]) < 1e-5 * r["grad_l2"] * dn, (b, i)
            if r["fd"][i] is not None:
                gap_gpu = abs(gd - r["fd"][i]) / (gn * dn)
                gap_oracle = abs(r["grad_dot_dir"][i] - r["fd"][i]) / (r["grad_l2"] * dn)
                assert gap_oracle < 2e-2, (b, i, gap_oracle)
                assert abs(gap_gpu - gap_oracle) <= 0.1 * gap_oracle + 1e-5, (b, i, gap_gpu, gap_oracle)
    assert sum(r["fd"][0] is not None for r in ref["members"]) == len(mg.C4_FD_MEMBERS)
