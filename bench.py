#!/usr/bin/env python
"""Benchmark of the PDE-EPDiff LDDMM hot path on GB300.

Headline: Gauss-Newton Hessian-vector products per second at 128^3 (the
128^3 nested-ellipsoid registration workload: nt = 10, K = (Id - 0.005 Lap)^-2,
FP32 transport / shooting / K-apply, FP64 reductions).  One step is one Hv:
forward Jacobi sweep over the stored time states, Gauss-Newton source,
adjoint Jacobi sweep and assembly, through the C ABI, inputs resident in HBM.
The line also reports the same metric end to end with host buffers, the
plain FP64 method, one full registration of the workload, the roofline of
the dominant kernel class, and the FP64 CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With N > 1 (torchrun) every rank runs an independent replica (one
registration does not shard without an all-to-all transpose per FFT pass),
and value is the Hv of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GN Hessian-vector products/s at 128^3"
UNIT = "Hv/s"
N128 = (128, 128, 128)
NT = 10
ALPHA = 0.005
WORKLOAD = ("128^3 registration workload: 3 nested random ellipsoids (0.2/0.5/0.9) + noise 0.02, "
            "target warped by a random |k|<=6 v0 (6 voxels), nt=10, K=(Id-0.005 Lap)^-2, weight 1e-3, "
            "Catmull-Rom SL transport, V metric, FP32 form with FP64 reductions")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--registrations", type=int, default=1, help="full registrations to time (0: skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-prof", action="store_true", help="skip the per-kernel profiled pass")
    ap.add_argument("--n", type=int, default=128, help="cubic grid size (profiling runs; the metric is 128)")
    ap.add_argument("--nt", type=int, default=NT, help="time steps (profiling runs; the metric uses 10)")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="requests of the serving trace, a prefix of its 256 (0: skip)")
    ap.add_argument("--no-plain-registration", action="store_true",
                    help="skip the registration of the workload with the plain FP64 method")
    ap.add_argument("--serve-fp64", type=int, default=2,
                    help="run the first M serving requests serially with the plain FP64 method and with the "
                         "FP32 form (0: skip)")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 256x300x256 registration (FP32, bfloat16 states, checkpointing)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- replicas
def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks of the default process group (x itself
    without one).  Timings use it: the job's time is its slowest replica."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput of `world` independent replicas (units per second)."""
    return world * units_per_rank / (ms_max / 1000.0)


# ----------------------------------------------------------------------------- inputs
def workload_inputs(n=N128, seed=1):
    """Phantom, true velocity and noise for the 128^3 workload (seeded)."""
    n = tuple(n)
    from paper_1807_04638_gb300 import synth
    P, v0, e0, e1 = synth.ellipsoid_pair_inputs(n, seed, kmax=6, max_disp_vox=6.0, noise_sigma=0.02)
    d = synth.band_limited_field(n, synth.rng_for(seed + 1000), 6.0, 3) * (2 * 3.141592653589793 / n[0])
    return P, v0, e0, e1, d


# DRAM traffic per launch of the stage kernels, from an ncu capture
# (profiles/fused_stages_128cubed_f32_ncu.md; one launch is one stage over the
# whole grid, the same at every nt), valid only for the kernel sources it was
# measured on: reported as null once the sources change.
TRAFFIC = {"digest": "d02ac607bd11f0f5", "adjoint_stage_fused": 359.7e6, "tangent_stage_fused": 386.5e6}


def kernel_digest():
    """Digest of the pass and stage-kernel sources (the dominant kernel
    classes and their job layout): a stored DRAM-traffic figure holds only
    for this digest."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1807_04638_gb300", "csrc")
    for f in ("common.cuh", "fft_fast.cuh", "fft_kernels.cuh", "fused_stage.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- serving workload
SERVE_SIZES = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (160, 192, 160)]


def serve_trace_inputs(nreq, seed=100):
    """Serving workload: exponential inter-arrival times (mean 0.25 s), grid
    ~ U{64^3, 96^3, 128^3, 160x192x160}, phantom ~ U{blob, ellipsoid}, a true
    velocity with the phantom's band and a peak displacement of n_min/20
    voxels.  Returns per request (arrival, shape, phantom, v0_true, noise0,
    noise1); targets are made by the caller's own shoot."""
    import numpy as np
    from paper_1807_04638_gb300 import synth
    rng = synth.rng_for(seed)
    t = 0.0
    out = []
    for i in range(nreq):
        t += rng.exponential(0.25)
        n = SERVE_SIZES[int(rng.integers(0, len(SERVE_SIZES)))]
        kind = int(rng.integers(0, 2))
        sub = synth.rng_for(seed * 1000 + i)
        disp = min(n) / 20.0
        if kind == 0:
            P = synth.blob_phantom(n, sub)
            v = synth.random_velocity(n, sub, 4, disp)
        else:
            P = synth.ellipsoid_phantom(n, sub)
            v = synth.random_velocity(n, sub, 6, disp)
        e0 = synth.noise(n, sub, 0.02)
        e1 = synth.noise(n, sub, 0.02)
        out.append((t, n, P, v, e0, e1))
    return out


def run_serving(args, dev):
    """Serve the trace in the FP32 form through the continuous-batching server
    (80 GB budget), optionally replay the first M requests serially in FP64."""
    import numpy as np
    import torch

    import paper_1807_04638_gb300 as pkg
    from paper_1807_04638_gb300.serve import Request, Server, latency_stats, serial
    trace = serve_trace_inputs(args.serve_requests)
    mk = lambda cd: pkg.default_params(alpha=ALPHA, nt=NT, compute_dtype=cd, state_dtype=cd, gn_maxit=8,
                                       pcg_maxit=20, pcg_rtol=0.1)
    p32 = mk(pkg.LDDMM_F32)
    reqs = []
    targets = {}
    for i, (t, n, P, v, e0, e1) in enumerate(trace):  # targets with the library's own shoot (untimed)
        if n not in targets:
            targets[n] = pkg.Handle(n, p32, device=dev.index)
        h = targets[n]
        m1 = h.new_img()
        T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
        h.lddmm_shoot(T(v), T(P), m1)
        I1 = m1.double().cpu().numpy() + e1
        reqs.append(Request(rid=i, I0=P + e0, I1=I1, params=p32, arrival=t))
    for h in targets.values():
        h.close()
    torch.cuda.empty_cache()
    srv = Server(budget_bytes=80e9, max_inflight=8, device=dev.index)
    try:
        res = srv.run_trace(reqs)
    finally:
        srv.close()
    st = latency_stats(res)
    out = {"requests": len(reqs), "budget_gb": 80, "offered_rate_per_s": 4.0,
           "sizes": [list(r.I0.shape) for r in reqs],
           "peak_inflight": srv.peak_inflight, "peak_workspace_gb": round(srv.peak_used / 1e9, 2),
           "mse_rel_mean": float(np.mean([r.report["mse_rel"] for r in res if r.report])), **st}
    if args.serve_fp64 > 0:
        # the plain FP64 method and the FP32 form, each serially in FIFO
        # order, on the first m requests of the trace
        m = min(args.serve_fp64, len(reqs))
        runs = {}
        for name, prm_ in (("plain_fp64_serial", mk(pkg.LDDMM_F64)), ("fp32_serial", p32)):
            sub = [Request(rid=r.rid, I0=r.I0, I1=r.I1, params=prm_, arrival=0.0) for r in reqs[:m]]
            t0 = time.perf_counter()
            ser = serial(sub, device=dev.index)
            runs[name] = (ser, time.perf_counter() - t0)
        served_sub = [r for r in res[:m] if r.report]
        for name, (ser, wall) in runs.items():
            ok = [r for r in ser if r.report]
            dm = [abs(a.report["mse_rel"] - b.report["mse_rel"]) / b.report["mse_rel"]
                  for a, b in zip(res[:m], ser) if a.report and b.report]
            out[name] = {"requests": m, "sizes": [list(r.I0.shape) for r in reqs[:m]],
                         "registrations_per_s": len(ok) / wall, "mean_latency_s": wall / max(len(ok), 1),
                         "mse_rel_mean": float(np.mean([r.report["mse_rel"] for r in ok])),
                         "served_fp32_mse_rel_mean_same_requests":
                             float(np.mean([r.report["mse_rel"] for r in served_sub])),
                         "max_rel_diff_mse_rel_vs_served": max(dm) if dm else None}
    return out


# ----------------------------------------------------------------------------- 256x300x256
N3 = (256, 300, 256)
C3_PCG_CAP = 10


def run_config3(dev, stream):
    """Register the brain-shaped 256x300x256 volume (perturbed nested
    ellipsoids with a 4-voxel boundary perturbation, noise 0.02; target =
    the phantom shot by a |k| <= 8, 8-voxel velocity plus noise) in the FP32
    form with bfloat16 stored states and forward states checkpointed every 2
    steps: 10 Gauss-Newton iterations, PCG rtol 0.1, at most 10 PCG iterations
    each (the bench's time budget; the configuration's cap of 50 takes about
    five minutes)."""
    import numpy as np
    import torch

    import paper_1807_04638_gb300 as pkg
    from paper_1807_04638_gb300 import synth
    P, v0t, e0, e1 = synth.ellipsoid_pair_inputs(N3, 2, kmax=8, max_disp_vox=8.0, noise_sigma=0.02,
                                                 perturb_vox=4.0)
    prm = pkg.default_params(alpha=ALPHA, nt=NT, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_BF16,
                             checkpoint_every=2, gn_maxit=10, pcg_maxit=C3_PCG_CAP, pcg_rtol=0.1)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    h = pkg.Handle(N3, prm, stream=stream, device=dev.index)
    try:
        m1 = h.new_img()
        h.lddmm_shoot(T(v0t), T(P), m1)  # target (untimed)
        I1 = (m1 + T(e1)).contiguous()
        I0 = T(P + e0)
        v = torch.zeros((3,) + N3, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = h.lddmm_register(I0, I1, v)
        torch.cuda.synchronize(dev)
        secs = time.perf_counter() - t0
    finally:
        h.close()
    return {"grid": list(N3), "form": "FP32, bfloat16 stored states, checkpoint every 2 steps", "seconds": secs,
            "weight": prm.weight, "pcg_rtol": 0.1, "pcg_cap": C3_PCG_CAP,
            "workspace_gb": round(pkg.workspace_bytes(N3, prm) / 1e9, 2), "gn_iters": r["gn_iters"],
            "pcg_iters_total": r["pcg_iters_total"], "mse_rel": r["mse_rel"], "gnorm_rel": r["gnorm_rel"],
            "jac_min": r["jac_min"], "jac_max": r["jac_max"], "status": r["status"]}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_hv_sample(P, v0, d, stages=2):
    """Time the FP64 oracle on a bounded sample of one Hv at 128^3: `stages`
    forward Jacobi stages and as many adjoint stages at a fixed linearisation
    state; scaled by 2 nt / stages to one Hv (a Hv is 2 nt of each)."""
    import numpy as np
    from oracle import lddmm_oracle as O
    g = O.Grid(N128, alpha=ALPHA)
    v = 0.5 * v0
    xi = 0.1 * d
    t0 = time.perf_counter()
    for _ in range(stages):
        be, bx = O.jacobi_A(g, v, d, xi)
        O.jacobi_A_T(g, v, be, bx)
    dt = time.perf_counter() - t0
    sec_per_hv = dt * (2 * NT) / stages
    return 1.0 / sec_per_hv, dt


def cpu_cores_used():
    return 1  # numpy's pocketfft and the elementwise work run on one thread


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_hv_measured(P, v0, d, workers):
    """One complete FP64 oracle Hv at 128^3 (tangent sweep, Gauss-Newton
    source, adjoint sweep and assembly: O.hessvec), timed with its
    transforms on `workers` threads (scipy.fft).  The linearisation point is
    the EPDiff trajectory of v0 / 2, computed untimed without the map
    transport, with the image at t = 1 taken as the phantom: the Hv's work
    does not depend on those values."""
    from oracle import lddmm_oracle as O
    g = O.Grid(N128, alpha=ALPHA)
    p = O.Params(alpha=ALPHA, nt=NT, weight=1e-3)
    O.set_fft_workers(workers)
    try:
        tr = O.shoot(g, 0.5 * v0, NT, P, transport=False)
        t0 = time.perf_counter()
        O.hessvec(g, p, tr, d)
        secs = time.perf_counter() - t0
    finally:
        O.set_fft_workers(None)
    return 1.0 / secs, secs


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import lddmm_oracle as O
    P, v0, e0, e1, d = workload_inputs()
    cores = host_cores()
    O.set_fft_workers(cores)
    try:
        for _ in range(args.warmup):
            oracle_hv_sample(P, v0, d, stages=1)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, _ = oracle_hv_sample(P, v0, d, stages=1)
            vals.append(v)
        wall = time.perf_counter() - t0
    finally:
        O.set_fft_workers(None)
    value = args.steps / sum(1.0 / v for v in vals)
    sample = ("per step: one forward Jacobi stage + one adjoint Jacobi stage of the FP64 NumPy oracle at 128^3 "
              f"(fixed linearisation state; transforms on {cores} threads through scipy.fft), scaled by "
              "2*nt = 20 to one Hv")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": list(N128), "nt": NT},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- native arm
def run_native(args, rank, world):
    import numpy as np
    import torch

    import paper_1807_04638_gb300 as pkg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = world > 1
    if dist:
        import torch.distributed as td

    def barrier():
        if dist:
            td.barrier()

    NG = (args.n,) * 3
    P, v0t, e0, e1, d = workload_inputs(NG)
    f32 = torch.float32
    T = lambda a, dt=f32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    prm = pkg.default_params(alpha=ALPHA, nt=args.nt, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32,
                             gn_maxit=10, pcg_maxit=50, pcg_rtol=0.1)
    stream = torch.cuda.current_stream(dev)
    h = pkg.Handle(NG, prm, stream=stream, device=dev.index)
    # target: phantom warped by the true velocity (library shoot), plus noise
    I0 = T(P + e0)
    m1 = h.new_img()
    h.lddmm_shoot(T(v0t), T(P), m1)
    I1 = (m1 + T(e1)).contiguous()
    v0 = T(0.5 * v0t)
    grad = h.new_vec()
    h.lddmm_gradient(v0, I0, I1, grad, energy=True)
    delta = T(d)
    hv = h.new_vec()

    # ---- device-resident timing
    for _ in range(args.warmup):
        h.lddmm_hessvec(delta, hv)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(dev.index)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        h.lddmm_hessvec(delta, hv)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    value = replica_throughput(args.steps, world, ms)
    hv_host = hv.double().cpu().numpy()
    finite = bool(np.isfinite(hv_host).all())

    # ---- end to end through the public API with pinned host buffers
    e2e_value, vec_bytes = None, 3 * int(np.prod(NG)) * 4
    if not args.no_e2e:
        e2e_value = e2e_run(args, h, d, hv, stream, dev, barrier, world, dist)
    out_e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": vec_bytes, "d2h_bytes_per_step": vec_bytes}

    # ---- kernel classes: CUDA events around every launch (separate pass)
    roofline, shares, launches_per_hv = None, None, None
    if not args.no_prof:
        roofline, shares, launches_per_hv = profile_run(h, delta, hv, value, world)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if NG == N128 and args.nt == NT else f"{NG} nt={args.nt} profiling case",
                   "n": list(NG), "nt": args.nt,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2_policy": "inputs larger than L2: 4.0 GB of stored time states read per Hv"},
        "clocks": clocks,
        "e2e": out_e2e,
        "gpu_launches": int(round(launches_per_hv * args.steps)) if launches_per_hv else None,
        "roofline": roofline,
        "kernel_shares": shares,
        "result_finite": finite,
    }
    # the characterisations beside the headline (precision and solver forms,
    # serving, CPU baseline) run at N = 1 only, so a multi-GPU run holds its
    # GPUs for the timed work alone
    if world > 1:
        args.no_fp64, args.no_cpu = True, True
        args.registrations, args.serve_requests = 0, 0
    return finish(args, out, h, v0t, d, I0, I1, stream, dev, rank, P, NG)


def e2e_run(args, h, d, hv, stream, dev, barrier, world, dist):
    import numpy as np
    import torch
    f32 = torch.float32
    hd = torch.tensor(np.ascontiguousarray(d), dtype=f32).pin_memory()
    ho = torch.empty_like(hd).pin_memory()
    dbuf = h.new_vec()
    for _ in range(2):
        dbuf.copy_(hd, non_blocking=True)
        h.lddmm_hessvec(dbuf, hv)
        ho.copy_(hv, non_blocking=True)
    torch.cuda.synchronize(dev)
    barrier()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    for _ in range(args.steps):
        dbuf.copy_(hd, non_blocking=True)
        h.lddmm_hessvec(dbuf, hv)
        ho.copy_(hv, non_blocking=True)
    ee1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ems = max_over_ranks(ee0.elapsed_time(ee1), dev)
    return replica_throughput(args.steps, world, ems)


def profile_run(h, delta, hv, value, world):
    h.lddmm_profile(True)
    nprof = 3
    for _ in range(nprof):
        h.lddmm_hessvec(delta, hv)
    prof = h.lddmm_profile_read()
    h.lddmm_profile(False)
    tot_ms = sum(v[0] for v in prof.values())
    launches_per_hv = sum(v[2] for v in prof.values()) / nprof
    dom = max(prof, key=lambda k: prof[k][0])
    dms, dbytes, dn = prof[dom]
    peak, peak_kind = load_peaks()
    achieved = (dbytes / dn) / ((dms / dn) / 1000.0) / 1e9 if dn else None
    shares = {k: {"share": round(v[0] / tot_ms, 4), "launches_per_hv": v[2] / nprof,
                  "gbs": round((v[1] / 1e9) / (v[0] / 1000.0), 1) if v[0] > 0 else None}
              for k, v in prof.items() if v[2] > 0}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1) if achieved else None,
                "peak": peak, "peak_kind": peak_kind + " hbm_gbs (STREAM-style copy)", "unit": "GB/s",
                "frac": round(achieved / peak, 4) if achieved else None,
                "traffic": TRAFFIC.get(dom) if TRAFFIC["digest"] == kernel_digest() else None,
                "kernel_digest": kernel_digest(),
                "algorithmic_bytes_per_launch": dbytes / dn if dn else None,
                "path_frac_compulsory_5GB_per_hv": round(value / world * 5.0e9 / (peak * 1e9), 4)}
    return roofline, shares, launches_per_hv


def cufft_crosscheck(NG, dev, stream, reps=10):
    """K-apply of a 3-component FP32 field: lddmm_apply_metric (hand-written
    passes) vs torch.fft.rfftn / irfftn (cuFFT) with the same symbol; times
    (CUDA events, mean of `reps` after a warm-up) and relative difference."""
    import numpy as np
    import torch

    import paper_1807_04638_gb300 as pkg
    prm = pkg.default_params(alpha=ALPHA, nt=2, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_F32)
    h = pkg.Handle(NG, prm, stream=stream, device=dev.index)
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn((3,) + tuple(NG), generator=g, dtype=torch.float32).to(dev)
    ours = torch.empty_like(x)
    k = [torch.fft.fftfreq(n, d=1.0 / n, device=dev, dtype=torch.float64) for n in NG[:2]]
    k.append(torch.fft.rfftfreq(NG[2], d=1.0 / NG[2], device=dev, dtype=torch.float64))
    ksq = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
    Khat = (1.0 / (1.0 + ALPHA * ksq) ** 2).to(torch.float32)

    def lib_fft():
        return torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)) * Khat, s=tuple(NG), dim=(1, 2, 3))

    def timed(fn, st):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    ms_ours = timed(lambda: h.lddmm_apply_metric(x, ours, -1), stream)
    with torch.cuda.stream(stream):
        ms_lib = timed(lib_fft, stream)
        ref = lib_fft()
    torch.cuda.synchronize(dev)
    h.close()
    diff = float(torch.linalg.vector_norm((ours - ref).double()) / torch.linalg.vector_norm(ref.double()))
    return {"what": "K = (Id - 0.005 Lap)^-2 on 3 x 128^3 FP32 fields", "lddmm_apply_metric_ms": round(ms_ours, 4),
            "torch_fft_cufft_ms": round(ms_lib, 4), "rel_l2_diff": diff}


def finish(args, out, h, v0t, d, I0, I1, stream, dev, rank, P, NG):
    import numpy as np
    import torch

    import paper_1807_04638_gb300 as pkg
    f32 = torch.float32
    prm = h.params

    # ---- precision form: the same Hv with bfloat16 stored states
    if not args.no_fp64 and rank == 0:
        prmb = pkg.default_params(alpha=ALPHA, nt=args.nt, compute_dtype=pkg.LDDMM_F32, state_dtype=pkg.LDDMM_BF16)
        h.close()
        torch.cuda.empty_cache()
        hb = pkg.Handle(NG, prmb, stream=stream, device=dev.index)
        Tf = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=f32, device=dev)
        gb = hb.new_vec()
        hb.lddmm_gradient(Tf(0.5 * v0t), I0, I1, gb, energy=False)
        db, hvb = Tf(d), hb.new_vec()
        for _ in range(2):
            hb.lddmm_hessvec(db, hvb)
        torch.cuda.synchronize(dev)
        kb = 5
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(kb):
            hb.lddmm_hessvec(db, hvb)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        msb = b0.elapsed_time(b1) / kb
        out["bf16_states"] = {"value": 1000.0 / msb, "unit": UNIT, "ms_per_hv": msb, "steps": kb,
                              "workspace_gb": round(pkg.workspace_bytes(NG, prmb) / 1e9, 2),
                              "fp32_states_workspace_gb": round(pkg.workspace_bytes(NG, prm) / 1e9, 2)}
        hb.close()
        torch.cuda.empty_cache()

    # ---- plain FP64 method, same workload (a few Hv)
    if not args.no_fp64 and rank == 0:
        prm64 = pkg.default_params(alpha=ALPHA, nt=args.nt)
        h64 = pkg.Handle(NG, prm64, stream=stream, device=dev.index)
        D = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        g64 = h64.new_vec()
        h64.lddmm_gradient(D(0.5 * v0t), I0.double(), I1.double(), g64, energy=False)
        d64, hv64 = D(d), h64.new_vec()
        h64.lddmm_hessvec(d64, hv64)
        torch.cuda.synchronize(dev)
        k64 = 3
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(k64):
            h64.lddmm_hessvec(d64, hv64)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = a0.elapsed_time(a1) / k64
        out["plain_fp64"] = {"value": 1000.0 / ms64, "unit": UNIT, "ms_per_hv": ms64, "steps": k64}
        # what bounds it: the FP64 FMA rate (measured by the probe kernel) vs
        # the FFT passes' achieved bandwidth
        if not args.no_prof:
            _, sh64, _ = profile_run(h64, d64, hv64, 1000.0 / ms64, 1)
            out["plain_fp64"]["kernel_shares"] = sh64
        out["plain_fp64"]["fp64_fma_tflops_measured"] = round(pkg.probe_fp64_fma(dev.index), 3)
        h64.close()
        del h64
        torch.cuda.empty_cache()

    # ---- one reduced gradient per mode: Jacobi-field (Sec. 3) and the exact
    # gradient of the discrete energy (transposed transport)
    if not args.no_fp64 and rank == 0:
        gm = {}
        for name, mode in (("jacobi", pkg.LDDMM_GRAD_JACOBI), ("discrete", pkg.LDDMM_GRAD_DISCRETE)):
            prmg = pkg.default_params(**{f: getattr(prm, f) for f, _ in prm._fields_})
            prmg.gradient_mode = mode
            hg = pkg.Handle(NG, prmg, stream=stream, device=dev.index)
            vg, gg = torch.tensor(0.5 * v0t, dtype=f32, device=dev), hg.new_vec()
            hg.lddmm_gradient(vg, I0, I1, gg, energy=False)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                hg.lddmm_gradient(vg, I0, I1, gg, energy=False)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            gm[name + "_ms"] = round(e0.elapsed_time(e1) / 3, 3)
            hg.close()
        out["gradient"] = gm

    # ---- cuFFT cross-check of the K-apply: the library FFT (torch.fft) timed
    # beside the hand-written passes on the same 3-component 128^3 FP32 field
    if not args.no_fp64 and rank == 0:
        out["cufft_crosscheck"] = cufft_crosscheck(NG, dev, stream)

    # ---- full registrations of the workload (FP32 form).  The headline runs
    # at regularisation weight 1e-2, where the map stays diffeomorphic (min
    # det J > 0) on this noisy workload; at 1e-3 the solution folds, and the
    # FP32 trajectory then depends on rounding (reported beside it).
    def register(prm_r, dtype=f32, runs=1):
        hr = pkg.Handle(NG, prm_r, stream=stream, device=dev.index)
        lat, rep = [], None
        for _ in range(runs):
            v = torch.zeros((3,) + NG, dtype=dtype, device=dev)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rep = hr.lddmm_register(I0.to(dtype), I1.to(dtype), v)
            torch.cuda.synchronize(dev)
            lat.append(time.perf_counter() - t0)
        hr.close()
        keys = ("gn_iters", "pcg_iters_total", "mse_rel", "gnorm_rel", "jac_min", "jac_max", "status")
        return sorted(lat), {k: rep[k] for k in keys}

    def with_(**kw):
        p_ = pkg.default_params(**{f: getattr(prm, f) for f, _ in prm._fields_})
        for k, v in kw.items():
            setattr(p_, k, v)
        return p_

    W_HEAD = 1e-2
    if args.registrations > 0 and rank == 0:
        lat, rep = register(with_(weight=W_HEAD), runs=args.registrations)
        q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
        out["registration"] = {"weight": W_HEAD, "registrations_per_s": len(lat) / sum(lat), "p50_s": q(0.5),
                               "p99_s": q(0.99), "runs": len(lat), **rep}
        # the paper's two variants side by side: PCG stopping and the reported
        # gradient norm in the L2 metric instead of V
        lat, rep = register(with_(weight=W_HEAD, space=pkg.LDDMM_SPACE_L2))
        out["registration_l2_variant"] = {"weight": W_HEAD, "seconds": lat[0], **rep}
        # weight 1e-3: the map folds (min det J < 0), and builds whose Hv
        # agree with the FP64 method equally well reach different solutions
        lat, rep = register(with_(weight=1e-3))
        out["registration_w1e-3"] = {"weight": 1e-3, "seconds": lat[0], **rep,
                                     "note": "folding regime: the FP32 trajectory depends on rounding"}

    # ---- the headline registration with the plain FP64 method
    if not args.no_plain_registration and args.registrations > 0 and rank == 0:
        lat, rep = register(with_(weight=W_HEAD, compute_dtype=pkg.LDDMM_F64, state_dtype=pkg.LDDMM_F64),
                            dtype=torch.float64)
        out["registration_plain_fp64"] = {"weight": W_HEAD, "seconds": lat[0], **rep}

    # ---- the 256x300x256 brain-shaped volume: FP32, bfloat16 states,
    # checkpointed forward states, 10 Gauss-Newton iterations
    if not args.no_config3 and args.registrations > 0 and rank == 0:
        out["registration_256x300x256"] = run_config3(dev, stream)

    # ---- serving trace (continuous batching, mixed grid sizes)
    if args.serve_requests > 0 and rank == 0:
        out["serving"] = run_serving(args, dev)

    # ---- CPU oracle on the host cores: one complete Hv on every core, and a
    # single-thread sample of Jacobi stages
    if not args.no_cpu and rank == 0 and tuple(NG) == N128:
        cores = host_cores()
        mv, msecs = oracle_hv_measured(P, v0t, d, cores)
        cv, secs = oracle_hv_sample(P, v0t, d, stages=2)
        out["cpu_baseline"] = {"value": mv, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "host_cores": os.cpu_count(),
                               "sample": f"one complete FP64 NumPy oracle Hv at 128^3, nt = 10 ({msecs:.1f} s), "
                                         f"transforms on {cores} threads (scipy.fft), measured once",
                               "single_thread": {"value": cv, "unit": UNIT, "cores": 1,
                                                 "sample": f"2 forward + 2 adjoint Jacobi stages at 128^3 "
                                                           f"({secs:.1f} s, numpy.fft), scaled by 2*nt/2 = 10 "
                                                           f"to one Hv"}}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "native":
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(dev)
        # the handles and the tensors around them live on a stream of their
        # own, as a user's would: the legacy default stream cannot be captured,
        # so the Hessian-vector product's CUDA graph needs another stream
        with torch.cuda.stream(torch.cuda.Stream(dev)):
            run_native(args, rank, world)
    if world > 1 and args.impl == "native":
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
