"""Particle-sharded k-space force across ranks (the exchange of Sec. 2.4's O(1)
communication): every rank draws the same batch, sums its own particles' structure
factors and charge sums, one allreduce of P x 4 + 4 float64 forms the totals, and each
rank evaluates the forces of its own particles from them.

Only the exchange lives here; the arithmetic runs in librbe2d (CudaShardBackend) or in
whatever backend a caller provides with the same four methods.
"""
from __future__ import annotations

import torch

from . import binding as B


class CudaShardBackend:
    """The four steps of a sharded evaluation on one rank's RBE2D context."""

    def __init__(self, model, flags=B.RBE2D_KSPACE | B.RBE2D_IBC):
        self.m = model
        self.flags = flags

    def sample(self, step):
        B.rbe2d_sample_k(self.m.ctx, step, None)

    def partial(self, pos, q):
        pos, q, fl = self.m._inputs(pos, q)
        self._in = (pos, q, fl)
        rho = torch.empty((self.m.P, 4), dtype=torch.float64, device=self.m.device)
        sums = torch.empty(4, dtype=torch.float64, device=self.m.device)
        B.rbe2d_structure_factor(self.m.ctx, q.shape[0], pos, q, fl, rho)
        B.rbe2d_charge_sums(self.m.ctx, sums)
        return rho, sums

    def set_totals(self, rho, sums):
        pos, q, _ = self._in
        B.rbe2d_set_structure_factor(self.m.ctx, q.shape[0], rho.contiguous(), sums.contiguous())

    def force(self, pos, q):
        pos, q, fl = self._in
        F = torch.empty((q.shape[0], 3), dtype=self.m.out_dtype, device=self.m.device)
        B.rbe2d_force(self.m.ctx, q.shape[0], pos, q, self.flags | fl | B.RBE2D_REUSE_SF, F)
        return F


class ShardedEvaluator:
    """force(pos_local, q_local, step): this rank's forces of a system split over the
    ranks of `group`; `allreduce` defaults to torch.distributed.all_reduce (sum)."""

    def __init__(self, backend, group=None, allreduce=None):
        self.backend = backend
        self.group = group
        if allreduce is None:
            import torch.distributed as dist
            allreduce = lambda t: dist.all_reduce(t, group=self.group)
        self.allreduce = allreduce

    def force(self, pos, q, step):
        self.backend.sample(step)
        rho, sums = self.backend.partial(pos, q)
        P = rho.shape[0]
        buf = torch.cat([rho.reshape(-1).to(torch.float64), sums.reshape(-1).to(torch.float64)])
        self.allreduce(buf)  # the one exchange: P x 4 + 4 doubles
        self.backend.set_totals(buf[: 4 * P].reshape(P, 4), buf[4 * P:])
        return self.backend.force(pos, q)
