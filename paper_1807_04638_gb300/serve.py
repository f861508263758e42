"""Continuous-batching registration server on one GPU.

Requests (source, target, grid, parameters) arrive at any time.  The
scheduler admits a waiting request as soon as a slot is free and the device
memory it needs fits in the HBM budget, counting every live handle's
workspace with ``lddmm_workspace_bytes``.  Each admitted request runs its
whole inexact Gauss-Newton-Krylov registration (``lddmm_register``) on its
own handle and CUDA stream from a worker thread (the ctypes call releases the
GIL), so the registrations in flight overlap on the device.  A handle keeps
its stored time states and PCG vectors on the device for the life of its
registration and is then parked for reuse by the next request of the same
shape; parked handles are destroyed when another shape needs the memory.

Requests that can never fit the budget, or that carry invalid or non-finite
data, fail with an error status; the others are unaffected.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import _native as N


@dataclasses.dataclass
class Request:
    rid: int
    I0: np.ndarray                    # [n0, n1, n2] host array
    I1: np.ndarray
    params: N.lddmm_params
    lengths: Optional[Tuple[float, float, float]] = None
    arrival: float = 0.0              # seconds since the trace start
    deadline_s: Optional[float] = None  # host watchdog: fail if not admitted in time


@dataclasses.dataclass
class Result:
    rid: int
    status: str
    v0: Optional[np.ndarray] = None
    report: Optional[dict] = None
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _key(n, p: N.lddmm_params, lengths):
    # a parked handle is reused only for exactly the same grid and parameters
    return (tuple(n), tuple(lengths) if lengths else None) + tuple(getattr(p, f) for f, _ in p._fields_)


@dataclasses.dataclass
class Reservation:
    """Bytes counted against the budget for a handle not created yet, and the
    parked handles evicted to make room, which the caller closes (outside the
    server's lock, since closing and creating handles call into CUDA)."""
    need: int
    victims: List[object]


class HandlePool:
    """HBM-budget accounting of the live handles of a server: the ones in
    use and the ones parked for reuse by a later request with the same key
    (grid and parameters).  A handle is a pair (object with close(), bytes).
    The pool itself takes no lock; the server calls it under its own, and
    creates and closes handles outside it."""

    def __init__(self, budget_bytes: float):
        self.budget = float(budget_bytes)
        self.used = 0.0                        # bytes of live handles (busy + parked)
        self.peak_used = 0.0
        self.parked: Dict[tuple, List[Tuple[object, int]]] = {}

    def reserve(self, key, need: int):
        """A parked handle of `key` as (handle, bytes), else a Reservation of
        `need` bytes once they fit the budget, evicting parked handles of
        other keys to make room.  None when the request must wait for handles
        in use to be released; raises ValueError when it can never fit."""
        pool = self.parked.get(key)
        if pool:
            return pool.pop()
        if need <= 0:
            raise ValueError("invalid request shape or parameters")
        if need > self.budget:
            raise ValueError(f"exceeds the HBM budget ({need / 1e9:.1f} GB > {self.budget / 1e9:.1f} GB)")
        evicted = []  # (key, handle, bytes)
        while self.used + need > self.budget:
            victim = next((kk for kk, v in self.parked.items() if v), None)
            if victim is None:
                # not enough room yet: the evicted handles stay parked
                for kk, h, b in evicted:
                    self.parked[kk].append((h, b))
                    self.used += b
                return None
            h, b = self.parked[victim].pop()
            evicted.append((victim, h, b))
            self.used -= b
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        return Reservation(need, [h for _, h, _ in evicted])

    def cancel(self, r: Reservation):
        """The handle of a reservation could not be created."""
        self.used -= r.need

    def acquire(self, key, need: int, make):
        """reserve(), then close the evicted handles and create the new one
        with make() in the caller's thread.  Returns (handle, bytes) or None;
        raises ValueError when the request can never fit."""
        r = self.reserve(key, need)
        if not isinstance(r, Reservation):
            return r
        for h in r.victims:
            h.close()
        try:
            return make(), r.need
        except Exception:
            self.cancel(r)
            raise

    def park(self, key, hb):
        self.parked.setdefault(key, []).append(hb)

    def drop(self, hb):
        """Forget a handle that is not to be reused (its request failed); the
        caller closes it."""
        self.used -= hb[1]
        return hb[0]

    def close_parked(self):
        for pool in self.parked.values():
            for h, b in pool:
                h.close()
                self.used -= b
        self.parked.clear()


class Server:
    """Admission by HBM budget, one stream per in-flight registration."""

    def __init__(self, budget_bytes: float = 80e9, max_inflight: int = 8, device: int = 0):
        import torch
        self.torch = torch
        self.pool = HandlePool(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.device = torch.device("cuda", device)
        self.lock = threading.Condition()
        self.inflight = 0
        self.results: Dict[int, Result] = {}
        self.t0 = None
        self.threads: List[threading.Thread] = []
        self.peak_inflight = 0

    @property
    def peak_used(self) -> float:
        return self.pool.peak_used

    # -- memory accounting ------------------------------------------------------
    def _reserve_handle(self, req: Request):
        """Called with the lock held: a parked handle, a Reservation, or None
        if the request must wait."""
        n = req.I0.shape
        k = _key(n, req.params, req.lengths)
        return self.pool.reserve(k, N.workspace_bytes(n, req.params, req.lengths))

    def _make_handle(self, req: Request) -> N.Handle:
        """Called without the lock (from the request's worker thread)."""
        with self.torch.cuda.device(self.device):
            stream = self.torch.cuda.Stream(device=self.device)
            return N.Handle(req.I0.shape, req.params, lengths=req.lengths, stream=stream,
                            device=self.device.index)

    def _release_handle(self, req: Request, hb):
        self.pool.park(_key(req.I0.shape, req.params, req.lengths), hb)

    # -- request execution ------------------------------------------------------
    def _run(self, req: Request, hb):
        torch = self.torch
        res = self.results[req.rid]
        if isinstance(hb, Reservation):
            # evict and create outside the lock: other requests keep running
            # and releasing their handles meanwhile
            try:
                for victim in hb.victims:
                    victim.close()
                hb = (self._make_handle(req), hb.need)
            except Exception as e:
                res.status = f"error: {e}"
                res.finished = time.perf_counter() - self.t0
                with self.lock:
                    self.pool.cancel(hb)
                    self.inflight -= 1
                    self.lock.notify_all()
                return
        h, _ = hb
        try:
            dt = h.dtype
            if not (np.isfinite(req.I0).all() and np.isfinite(req.I1).all()):
                raise N.LddmmError(6, "request data")
            with torch.cuda.device(self.device), torch.cuda.stream(h.stream):
                I0 = torch.from_numpy(np.ascontiguousarray(req.I0)).to(self.device, dt, non_blocking=True)
                I1 = torch.from_numpy(np.ascontiguousarray(req.I1)).to(self.device, dt, non_blocking=True)
                v = torch.zeros((3,) + tuple(req.I0.shape), dtype=dt, device=self.device)
                rep = h.lddmm_register(I0, I1, v)
                res.v0 = v.double().cpu().numpy()
            res.report = rep
            res.status = rep["status"]
        except Exception as e:  # the request fails alone
            res.status = f"error: {e}"
        finally:
            res.finished = time.perf_counter() - self.t0
            sticky = N.lib().lddmm_last_status(h._h) if h._h else 0
            if sticky != 0:  # a failed handle is not reused; closed outside the lock
                h.close()
            with self.lock:
                if sticky != 0:
                    self.pool.drop(hb)
                else:
                    self._release_handle(req, hb)
                self.inflight -= 1
                self.lock.notify_all()

    def _admit_loop(self, pending: List[Request]):
        """Admit requests in arrival order as slots and memory free up."""
        i = 0
        backlog: List[Request] = []
        while i < len(pending) or backlog:
            now = time.perf_counter() - self.t0
            while i < len(pending) and pending[i].arrival <= now:
                backlog.append(pending[i])
                i += 1
            admitted_any = False
            with self.lock:
                while backlog and self.inflight < self.max_inflight:
                    req = backlog[0]
                    if req.deadline_s is not None and now - req.arrival > req.deadline_s:
                        backlog.pop(0)
                        r = self.results[req.rid]
                        r.status, r.finished = "error: admission deadline exceeded", now
                        continue
                    try:
                        hb = self._reserve_handle(req)
                    except Exception as e:
                        backlog.pop(0)
                        r = self.results[req.rid]
                        r.status, r.finished = f"error: {e}", now
                        continue
                    if hb is None:
                        if self.inflight == 0:   # can never fit
                            backlog.pop(0)
                            r = self.results[req.rid]
                            r.status, r.finished = "error: exceeds the HBM budget", now
                            continue
                        break
                    backlog.pop(0)
                    self.inflight += 1
                    self.peak_inflight = max(self.peak_inflight, self.inflight)
                    self.results[req.rid].admitted = now
                    t = threading.Thread(target=self._run, args=(req, hb), daemon=True)
                    self.threads.append(t)
                    t.start()
                    admitted_any = True
                if not admitted_any:
                    nxt = pending[i].arrival - now if i < len(pending) else 0.05
                    self.lock.wait(timeout=max(0.001, min(nxt, 0.05)))

    def run_trace(self, requests: List[Request]) -> List[Result]:
        """Play a trace (arrival times relative to now) and wait for every result."""
        self.t0 = time.perf_counter()
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            self.results[r.rid] = Result(rid=r.rid, status="pending", arrival=r.arrival)
        self._admit_loop(reqs)
        for t in self.threads:
            t.join()
        return [self.results[r.rid] for r in requests]

    def close(self):
        with self.lock:
            self.pool.close_parked()


def serial(requests: List[Request], device: int = 0) -> List[Result]:
    """The same requests one after another on one stream (baseline)."""
    srv = Server(budget_bytes=float("inf"), max_inflight=1, device=device)
    try:
        reqs = [dataclasses.replace(r, arrival=0.0) for r in requests]
        return srv.run_trace(reqs)
    finally:
        srv.close()


def latency_stats(results: List[Result]) -> dict:
    ok = [r for r in results if r.status in ("LDDMM_OK", "LDDMM_WARN_LINESEARCH")]
    lat = sorted(r.latency for r in ok)
    if not lat:
        return {"completed": 0}
    q = lambda p: float(np.percentile(lat, p))
    span = max(r.finished for r in ok) - min(r.arrival for r in ok)
    return {"completed": len(ok), "failed": len(results) - len(ok), "p50_s": q(50), "p99_s": q(99),
            "mean_s": float(np.mean(lat)), "registrations_per_s": len(ok) / span if span > 0 else None,
            "makespan_s": span}
