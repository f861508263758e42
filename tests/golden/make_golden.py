"""Writes the stored expected values under tests/golden/ by calling the FP64
oracle only (no GPU code).  Run from the repository root:

    python tests/golden/make_golden.py [config1] [bench128] [config4] [config3]

bench128_samples.json: the 128^3 benchmark workload (nested ellipsoids,
seed 1; target = the oracle's shoot of the true velocity plus noise; nt = 10,
K = (Id - 0.005 Lap)^-2, weight 1e-3, V metric): the energy, the L2 norms of
the V gradient and of the V Hessian-vector product at v0 = v0_true / 2 in
the direction of the workload, and their values at 2048 seeded sample
points (about 12 minutes of CPU).  bench128_planes.npz: complete planes of
the same two fields (BENCH128_HV_PLANES, BENCH128_GRAD_PLANES).

config1_register_32cubed.json: the plain-method registration of the 32^3
blob-phantom workload (seed 0; target = the oracle's shoot of a random
|k| <= 4 velocity with a 2-voxel peak displacement; nt = 10,
K = (Id - 0.01 Lap)^-2, weight 1e-3, 5 Gauss-Newton iterations of at most
10 PCG iterations, PCG relative tolerance 0.1, Catmull-Rom transport, V
metric): the oracle's energy trace, PCG counts, Armijo steps and final
metrics, plus the energy and gradient norm at v0 = 0.

config4_96cubed.json: the differentiation workload (8 x 96^3 blob pairs,
see C4_*): per member the loss, the gradient of ||m1 - I1||^2 with respect
to v0 at 2048 sample points, its norm and its projections on 16 directions,
and for four members central differences of the loss in those directions
(about 40 minutes on 6 cores).

config3_256x300x256.json, config3_planes.npz: the brain-shaped 256x300x256
grid (see C3_*): the oracle's shoot at nt = 2, u1 and m1 at 4096 sample
points, their norms, the kinetic energies, and complete planes stored in
single precision (C3_U_PLANES, C3_M_PLANES).
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


# complete planes (axis, index) of the 128^3 results stored beside the
# samples: x0 planes at a tile start and inside a tile, an x1 plane, the last
# x2 plane (the ragged end of the packed row pairs is none at 128, but the
# planes cross every tile of the other two axes)
BENCH128_HV_PLANES = ((0, 0), (0, 77), (1, 45), (2, 127))
BENCH128_GRAD_PLANES = ((0, 77), (2, 0))


def bench128():
    n, P, v0t, e0, e1, d, idx = bench128_inputs()
    g = O.Grid(n, alpha=0.005)
    p = O.Params(alpha=0.005, nt=10, weight=1e-3)
    I0 = P + e0
    m1t = O.shoot(g, v0t, p.nt, P).m1
    I1 = m1t + e1
    gl2, E, _, _, tr = O.gradient(g, p, 0.5 * v0t, I0, I1)
    gV = O.to_space(g, p, gl2)
    hV = O.to_space(g, p, O.hessvec(g, p, tr, d))
    out = {
        "what": "128^3 benchmark workload, FP64 oracle, v0 = v0_true / 2, V metric",
        "E": E, "grad_V_l2": float(np.linalg.norm(gV)), "hv_V_l2": float(np.linalg.norm(hV)),
        "idx": [int(i) for i in idx], "grad_V": [float(x) for x in gV.ravel()[idx]],
        "hv_V": [float(x) for x in hV.ravel()[idx]],
        # the noise-free target m1(P; v0_true): its norm and values at the
        # first 2048 scalar sample points (idx modulo n^3)
        "m1_true_l2": float(np.linalg.norm(m1t)),
        "m1_true": [float(x) for x in m1t.ravel()[idx % m1t.size]],
    }
    with open(os.path.join(HERE, "bench128_samples.json"), "w") as f:
        json.dump(out, f)
    planes = {}
    for name, field, cuts in (("hv_V", hV, BENCH128_HV_PLANES), ("grad_V", gV, BENCH128_GRAD_PLANES)):
        for axis, i in cuts:
            planes[f"{name}_axis{axis}_{i}"] = np.take(field, i, axis=1 + axis)
    np.savez_compressed(os.path.join(HERE, "bench128_planes.npz"), **planes)
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


# ---------------------------------------------------------------- config 4
# The differentiation workload: 8 independent 96^3 blob pairs (seeds 10..17,
# |k| <= 5, 3-voxel peak), nt = 10, K = (Id - 0.01 Lap)^-2; target = the
# oracle's shoot of the true velocity; evaluated at v0 = 0.6 v_true for the
# loss ||m1 - I1||^2 (plain sum over voxels).  16 directions per member:
# band-limited (|k| <= 5) fields of one voxel's length in grid RMS.
C4_N, C4_NT, C4_ALPHA = (96, 96, 96), 10, 0.01
C4_SEEDS = tuple(range(10, 18))
C4_NDIR, C4_FD_H = 16, 1e-4
C4_FD_MEMBERS = (0, 1, 2, 3)


def config4_member(b):
    """Inputs of batch member b: (I0, v_true, v0)."""
    I0, vt = synth.blob_pair_inputs(C4_N, C4_SEEDS[b], kmax=5, max_disp_vox=3.0)
    I0 = synth.spectral_gaussian_smooth(I0, 1.0)
    return I0, vt, 0.6 * vt


def config4_directions(b):
    r = synth.rng_for(3000 + b)
    h = 2 * np.pi / C4_N[0]
    return [synth.band_limited_field(C4_N, r, 5.0, 3) * h for _ in range(C4_NDIR)]


def config4_sample_idx():
    return synth.rng_for(4343).integers(0, 3 * int(np.prod(C4_N)), 2048)


def _c4_gradient(b):
    g = O.Grid(C4_N, alpha=C4_ALPHA)
    I0, vt, v0 = config4_member(b)
    I1 = O.shoot(g, vt, C4_NT, I0).m1
    tr = O.shoot(g, v0, C4_NT, I0)
    G = 2.0 * (tr.m1 - I1)
    grad = O.adjoint(g, tr, -G[None] * tr.grad_m1)
    idx = config4_sample_idx()
    return {"member": b, "loss": float(np.sum((tr.m1 - I1) ** 2)), "grad_l2": float(np.linalg.norm(grad)),
            "grad": [float(x) for x in grad.ravel()[idx]],
            "grad_dot_dir": [float(np.sum(grad * d)) for d in config4_directions(b)],
            "m1_true_l2": float(np.linalg.norm(I1)),
            "m1_true": [float(x) for x in I1.ravel()[idx % I1.size]]}, I1


def _c4_fd(args):
    b, i, I1 = args
    g = O.Grid(C4_N, alpha=C4_ALPHA)
    I0, _, v0 = config4_member(b)
    d = config4_directions(b)[i]
    L = lambda v: float(np.sum((O.shoot(g, v, C4_NT, I0).m1 - I1) ** 2))
    return b, i, (L(v0 + C4_FD_H * d) - L(v0 - C4_FD_H * d)) / (2 * C4_FD_H)


def config4(workers=6):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(_c4_gradient, range(len(C4_SEEDS)))
        members = [r for r, _ in res]
        I1s = {r["member"]: I1 for r, I1 in res}
        fds = pool.map(_c4_fd, [(b, i, I1s[b]) for b in C4_FD_MEMBERS for i in range(C4_NDIR)])
    for m in members:
        m["fd"] = [None] * C4_NDIR
    for b, i, v in fds:
        members[b]["fd"][i] = v
    out = {"what": "config-4 differentiation workload, 8 x 96^3, FP64 oracle: loss, gradient samples and "
                   "norm, gradient . direction and central differences (h = 1e-4) of the loss",
           "fd_members": list(C4_FD_MEMBERS), "members": members}
    with open(os.path.join(HERE, "config4_96cubed.json"), "w") as f:
        json.dump(out, f)
    print("config4 written")


# ---------------------------------------------------------------- config 3
# The brain-shaped 256x300x256 volume (perturbed nested ellipsoids, seed 2,
# |k| <= 8, 8-voxel peak; K = (Id - 0.005 Lap)^-2; each axis [0, 2 pi)):
# one short shoot (nt = 2, Catmull-Rom) of the true velocity from the noisy
# source.  The n1 = 300 axis runs the runtime-radix passes.
C3_N, C3_NT, C3_ALPHA = (256, 300, 256), 2, 0.005
C3_U_PLANES = ((0, 131), (2, 77))
C3_M_PLANES = ((1, 150),)


def config3_inputs():
    P, v0t, e0, _ = synth.ellipsoid_pair_inputs(C3_N, 2, kmax=8, max_disp_vox=8.0, noise_sigma=0.02,
                                                perturb_vox=4.0)
    return P + e0, v0t


def config3_sample_idx():
    return synth.rng_for(4444).integers(0, 3 * int(np.prod(C3_N)), 4096)


def config3():
    g = O.Grid(C3_N, alpha=C3_ALPHA)
    I0, v0t = config3_inputs()
    tr = O.shoot(g, v0t, C3_NT, I0)
    idx = config3_sample_idx()
    out = {"what": "config-3 grid 256x300x256, FP64 oracle shoot (nt = 2) of the true velocity",
           "u1_l2": float(np.linalg.norm(tr.u)), "m1_l2": float(np.linalg.norm(tr.m1)),
           "idx": [int(i) for i in idx], "u1": [float(x) for x in tr.u.ravel()[idx]],
           "m1": [float(x) for x in tr.m1.ravel()[idx % tr.m1.size]],
           "kinetic": [float(k) for k in tr.kinetic]}
    with open(os.path.join(HERE, "config3_256x300x256.json"), "w") as f:
        json.dump(out, f)
    planes = {}
    for axis, i in C3_U_PLANES:
        planes[f"u1_axis{axis}_{i}"] = np.take(tr.u, i, axis=1 + axis).astype(np.float32)
    for axis, i in C3_M_PLANES:
        planes[f"m1_axis{axis}_{i}"] = np.take(tr.m1, i, axis=axis).astype(np.float32)
    np.savez_compressed(os.path.join(HERE, "config3_planes.npz"), **planes)
    print("config3 written")


if __name__ == "__main__":
    which = sys.argv[1:] or ["config1", "bench128", "config4", "config3"]
    if "config1" in which:
        config1()
    if "bench128" in which:
        bench128()
    if "config4" in which:
        config4()
    if "config3" in which:
        config3()
