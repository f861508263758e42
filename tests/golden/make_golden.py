"""Writes the stored expected values under tests/golden/ by calling the FP64
oracle only (no GPU code).  Run from the repository root:

    python tests/golden/make_golden.py [config1] [bench128]

bench128_samples.json: the 128^3 benchmark workload (nested ellipsoids,
seed 1; target = the oracle's shoot of the true velocity plus noise; nt = 10,
K = (Id - 0.005 Lap)^-2, weight 1e-3, V metric): the energy, the L2 norms of
the V gradient and of the V Hessian-vector product at v0 = v0_true / 2 in
the direction of the workload, and their values at 2048 seeded sample
points (about 12 minutes of CPU).

config1_register_32cubed.json: the plain-method registration of the 32^3
blob-phantom workload (seed 0; target = the oracle's shoot of a random
|k| <= 4 velocity with a 2-voxel peak displacement; nt = 10,
K = (Id - 0.01 Lap)^-2, weight 1e-3, 5 Gauss-Newton iterations of at most
10 PCG iterations, PCG relative tolerance 0.1, Catmull-Rom transport, V
metric): the oracle's energy trace, PCG counts, Armijo steps and final
metrics, plus the energy and gradient norm at v0 = 0.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import lddmm_oracle as O  # noqa: E402
from paper_1807_04638_gb300 import synth  # noqa: E402


def config1_inputs():
    n, nt = (32, 32, 32), 10
    g = O.Grid(n, alpha=0.01)
    I0, vtrue = synth.blob_pair_inputs(n, 0, kmax=4, max_disp_vox=2.0)
    I1 = O.shoot(g, vtrue, nt, I0).m1
    return g, O.Params(alpha=0.01, nt=nt, weight=1e-3), I0, I1


def bench128_inputs():
    """The 128^3 workload's arrays (the same recipe and seeds as the
    benchmark) and the sample points."""
    from paper_1807_04638_gb300 import synth as S
    n = (128, 128, 128)
    P, v0t, e0, e1 = S.ellipsoid_pair_inputs(n, 1, kmax=6, max_disp_vox=6.0, noise_sigma=0.02)
    d = S.band_limited_field(n, S.rng_for(1 + 1000), 6.0, 3) * (2 * np.pi / n[0])
    idx = S.rng_for(4242).integers(0, 3 * int(np.prod(n)), 2048)
    return n, P, v0t, e0, e1, d, idx


def bench128():
    n, P, v0t, e0, e1, d, idx = bench128_inputs()
    g = O.Grid(n, alpha=0.005)
    p = O.Params(alpha=0.005, nt=10, weight=1e-3)
    I0 = P + e0
    I1 = O.shoot(g, v0t, p.nt, P).m1 + e1
    gl2, E, _, _, tr = O.gradient(g, p, 0.5 * v0t, I0, I1)
    gV = O.to_space(g, p, gl2)
    hV = O.to_space(g, p, O.hessvec(g, p, tr, d))
    out = {
        "what": "128^3 benchmark workload, FP64 oracle, v0 = v0_true / 2, V metric",
        "E": E, "grad_V_l2": float(np.linalg.norm(gV)), "hv_V_l2": float(np.linalg.norm(hV)),
        "idx": [int(i) for i in idx], "grad_V": [float(x) for x in gV.ravel()[idx]],
        "hv_V": [float(x) for x in hV.ravel()[idx]],
    }
    with open(os.path.join(HERE, "bench128_samples.json"), "w") as f:
        json.dump(out, f)
    print("bench128: E", E)


def config1():
    g, p, I0, I1 = config1_inputs()
    zero = np.zeros((3,) + g.n)
    g0, E0 = O.gradient(g, p, zero, I0, I1)[:2]
    rep = O.register(g, p, I0, I1, gn_maxit=5, pcg_maxit=10, pcg_rtol=0.1)
    out = {
        "what": "config-1 plain-method registration, 32^3, FP64 oracle",
        "E_at_zero": E0, "grad_L2_norm_at_zero": float(np.sqrt(g.dot(g0, g0))),
        "energies": rep.energies, "pcg_iters": rep.pcg_iters, "steps": rep.steps,
        "gnorm_rel": rep.gnorm_rel, "mse_rel": rep.mse_rel, "jac_min": rep.jac_min, "jac_max": rep.jac_max,
        "v0_l2_norm": float(np.sqrt(g.dot(rep.v0, rep.v0))),
    }
    with open(os.path.join(HERE, "config1_register_32cubed.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    which = sys.argv[1:] or ["config1", "bench128"]
    if "config1" in which:
        config1()
    if "bench128" in which:
        bench128()
