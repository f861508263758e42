"""Fused Jacobi stages (FP32 form): the kernels that run the axis-2 inverse
transform, the pointwise products and the axis-2 forward transform of a
tangent or adjoint stage in one pass give the results of the separate passes
(LDDMM_UNFUSED=1) to rounding, for every sweep product of the boundary, with
FP32 and bfloat16 stored states and the exact discrete gradient's extra
cotangents; the profiler shows which kernels ran.  Oracle parity of the same
outputs is covered by the parity tests, which run the fused path on every
grid whose three axes have register-blocked plans."""
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


def rel(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


CASES = [
    ((32, 32, 32), "f32", 4),
    ((64, 32, 128), "f32", 3),
    ((64, 64, 64), "bf16", 3),
    ((128, 128, 128), "f32", 2),
    ((32, 64, 256), "f32", 2),
]


@pytest.mark.parametrize("n,states,nt", CASES)
def test_fused_stages_equal_separate_passes(pkg, n, states, nt, monkeypatch):
    I0, vt = synth.blob_pair_inputs(n, 31, kmax=3, max_disp_vox=2.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = np.roll(I0, 1, axis=2)
    d = synth.band_limited_field(n, synth.rng_for(32), 4.0, 3) * (2 * np.pi / n[0])
    bx = synth.band_limited_field(n, synth.rng_for(33), 6.0, 3)
    be = synth.band_limited_field(n, synth.rng_for(34), 6.0, 3)
    sd = pkg.LDDMM_BF16 if states == "bf16" else pkg.LDDMM_F32
    # every workspace entry never written reads as NaN
    monkeypatch.setenv("LDDMM_POISON_WORKSPACE", "1")
    out = {}
    for mode in ("fused", "separate", "f64"):
        if mode == "separate":
            monkeypatch.setenv("LDDMM_UNFUSED", "1")
        else:
            monkeypatch.delenv("LDDMM_UNFUSED", raising=False)
        dt = torch.float64 if mode == "f64" else torch.float32
        T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
        if mode == "f64":
            prm = pkg.default_params(alpha=0.01, nt=nt)
        else:
            prm = pkg.default_params(alpha=0.01, nt=nt, compute_dtype=pkg.LDDMM_F32, state_dtype=sd)
        with pkg.Handle(n, prm) as h:
            r = {k: h.new_vec() for k in ("grad", "hv", "eta1", "xi1", "adj")}
            h.lddmm_profile(True)
            r["E"] = h.lddmm_gradient(T(0.5 * vt), T(I0), T(I1), r["grad"])[0]
            h.lddmm_hessvec(T(d), r["hv"])
            h.lddmm_jacobi_forward(T(d), r["eta1"], r["xi1"])
            h.lddmm_jacobi_adjoint(T(be), T(bx), r["adj"])
            h.lddmm_synchronize()
            prof = h.lddmm_profile_read()
            h.lddmm_profile(False)
            out[mode] = r
        launches = {k: v[2] for k, v in prof.items()}
        if mode == "fused":
            assert launches.get("tangent_stage_fused", 0) == 2 * nt * 2   # hessvec + jacobi_forward
            assert launches.get("adjoint_stage_fused", 0) == 2 * nt * 3   # gradient, hessvec, jacobi_adjoint
            assert launches.get("tangent_pointwise", 0) == 0 and launches.get("adjoint_pointwise", 0) == 0
        else:
            assert launches.get("tangent_stage_fused", 0) == 0 and launches.get("adjoint_stage_fused", 0) == 0
    f, s, ref = out["fused"], out["separate"], out["f64"]
    assert abs(f["E"] - s["E"]) <= 1e-12 * abs(s["E"])  # the shoot is the same kernels
    for k in ("grad", "hv", "eta1", "xi1", "adj"):
        # the two FP32 paths differ by rounding only: each is as close to the
        # FP64 engine's result as the other (L-weighted terms of the adjoint
        # amplify FP32 rounding in the high modes)
        ef, es = rel(f[k], ref[k]), rel(s[k], ref[k])
        assert ef <= 1.5 * es + 2e-7 and es <= 1.5 * ef + 2e-7, (k, ef, es)
        assert rel(f[k], s[k]) < 3e-5, (k, rel(f[k], s[k]))


def test_fused_adjoint_with_discrete_gradient_cotangents(pkg, monkeypatch):
    """The exact discrete gradient feeds real cotangents on eta into every
    transposed step; the fused adjoint stage adds them to its first group."""
    n, nt = (64, 64, 64), 4
    I0, vt = synth.blob_pair_inputs(n, 35, kmax=3, max_disp_vox=2.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    I1 = np.roll(I0, 1, axis=0)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    got = {}
    for mode in ("fused", "separate"):
        if mode == "separate":
            monkeypatch.setenv("LDDMM_UNFUSED", "1")
        else:
            monkeypatch.delenv("LDDMM_UNFUSED", raising=False)
        prm = pkg.default_params(alpha=0.01, nt=nt, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32,
                                 gradient_mode=pkg.LDDMM_GRAD_DISCRETE)
        with pkg.Handle(n, prm) as h:
            g = h.new_vec()
            h.lddmm_gradient(T(0.5 * vt), T(I0), T(I1), g)
            h.lddmm_synchronize()
            got[mode] = g
    # the transposed map steps scatter with atomics: rounding-level run-to-run noise
    assert rel(got["fused"], got["separate"]) < 1e-5
