"""Differentiable geodesic shooting: ``m1 = LddmmShoot.apply(v0, I0, shooter)``.

Forward: EPDiff shooting of each batch member's initial velocity and the
semi-Lagrangian warp of its source image (``lddmm_shoot``).  Backward: the
hand-written adjoint Jacobi sweep (``lddmm_shoot_vjp``): for an upstream
gradient G = d loss / d m1 the gradient with respect to v0 is
P T^T (-G grad m1), the reduced gradient of the paper carried from t = 1 back
to t = 0 (Sec. 3).  Gradients flow to v0 only; the source images are
treated as data.

Every batch member owns a handle (its stored time states are the backward's
linearisation point), created on its own CUDA stream so that the members'
sweeps overlap on the device; the Function orders those streams after the
caller's stream on entry and before it on exit.

Memory: with ``max_bytes`` the Shooter keeps every forward state while the
batch's workspaces fit, and otherwise stores the spectral velocity every 2
steps and recomputes the states segment by segment inside the backward
(checkpoint_every = 2: the smallest footprint, at one extra shoot per
backward whatever the segment length); the gradient is unchanged.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import _native as N


class Shooter:
    """Handles for a batch of ``batch`` registrations on one grid."""

    def __init__(self, n: Sequence[int], batch: int, params: Optional[N.lddmm_params] = None,
                 lengths=None, device=None, max_bytes: Optional[float] = None):
        self.n = tuple(int(x) for x in n)
        self.batch = int(batch)
        self.params = params if params is not None else N.default_params(
            compute_dtype=N.LDDMM_F32, state_dtype=N.LDDMM_F32)
        if max_bytes is not None:
            self.params = self.plan_memory(self.n, self.batch, self.params, max_bytes, lengths)
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(self.batch)]
        self.handles = [N.Handle(self.n, self.params, lengths=lengths, stream=s, device=dev.index)
                        for s in self.streams]
        self.dtype = self.handles[0].dtype

    @staticmethod
    def plan_memory(n, batch, params, max_bytes, lengths=None):
        """A copy of params that keeps every forward state if batch
        workspaces fit max_bytes, else checkpoints every 2 steps; raises
        MemoryError when even that does not fit."""
        p = N.default_params(**{f: getattr(params, f) for f, _ in params._fields_})
        if batch * N.workspace_bytes(n, p, lengths) <= max_bytes:
            return p
        if p.nt > 2:
            p.checkpoint_every = 2
            if batch * N.workspace_bytes(n, p, lengths) <= max_bytes:
                return p
        raise MemoryError(f"{batch} x {N.workspace_bytes(n, p, lengths) / 1e9:.2f} GB exceeds "
                          f"{max_bytes / 1e9:.2f} GB even with checkpointed states")

    def close(self):
        for h in self.handles:
            h.close()

    def _fork(self):
        cur = torch.cuda.current_stream(self.device)
        for s in self.streams:
            s.wait_stream(cur)

    def _join(self):
        cur = torch.cuda.current_stream(self.device)
        for s in self.streams:
            cur.wait_stream(s)


class LddmmShoot(torch.autograd.Function):
    """m1[b] = I0[b] o (phi_1^{v0[b]})^-1 for a batch; v0 [B,3,n0,n1,n2], I0 [B,n0,n1,n2]."""

    @staticmethod
    def forward(ctx, v0: torch.Tensor, I0: torch.Tensor, shooter: Shooter):
        B = v0.shape[0]
        if B != shooter.batch or v0.shape[1:] != (3,) + shooter.n or I0.shape != (B,) + shooter.n:
            raise ValueError("v0 must be [B,3,n0,n1,n2] and I0 [B,n0,n1,n2] for the shooter's batch and grid")
        v0c = v0.detach().to(shooter.dtype).contiguous()
        I0c = I0.detach().to(shooter.dtype).contiguous()
        m1 = torch.empty((B,) + shooter.n, dtype=shooter.dtype, device=v0.device)
        shooter._fork()
        for b, h in enumerate(shooter.handles):
            with torch.cuda.stream(shooter.streams[b]):
                h.lddmm_shoot(v0c[b], I0c[b], m1[b])
        shooter._join()
        for b in range(B):  # keep the inputs alive until the member streams are done
            v0c[b].record_stream(shooter.streams[b])
            I0c[b].record_stream(shooter.streams[b])
        ctx.shooter = shooter
        ctx.v0_dtype = v0.dtype
        return m1

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        shooter: Shooter = ctx.shooter
        Gc = G.detach().to(shooter.dtype).contiguous()
        B = Gc.shape[0]
        gv = torch.empty((B, 3) + shooter.n, dtype=shooter.dtype, device=Gc.device)
        shooter._fork()
        for b, h in enumerate(shooter.handles):
            with torch.cuda.stream(shooter.streams[b]):
                h.lddmm_shoot_vjp(Gc[b], gv[b])
        shooter._join()
        for b in range(B):
            Gc[b].record_stream(shooter.streams[b])
            gv[b].record_stream(shooter.streams[b])
        return gv.to(ctx.v0_dtype), None, None


def shoot(v0: torch.Tensor, I0: torch.Tensor, shooter: Shooter) -> torch.Tensor:
    """Differentiable batch shooting (see LddmmShoot)."""
    return LddmmShoot.apply(v0, I0, shooter)
