"""The sharded exchange on two CPU ranks (gloo, world size 2): the allreduced partial
structure factors and charge sums equal the whole system's, and each rank's forces equal
the whole-system forces of its particles.  The per-rank arithmetic is the FP64 oracle
(a test backend); what is under test is ShardedEvaluator's exchange."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleShardBackend:
    def __init__(self, s, pos_all, q_all, lo, hi, P, seed):
        import oracle as O
        self.O, self.s = O, s
        self.pos_all, self.q_all, self.lo, self.hi = pos_all, q_all, lo, hi
        self.P, self.seed = P, seed

    def sample(self, step):
        self.k = self.O.sample_k(self.s, self.seed, step, self.P)

    def partial(self, pos, q):
        rs = self.O.rho_sigma(self.s, pos.numpy(), q.numpy(), self.k)
        z = pos.numpy()[:, 2]
        sums = np.array([q.sum().item(), (q * q).sum().item(), float(np.sum(q.numpy() * z)), q.abs().sum().item()])
        return torch.as_tensor(rs), torch.as_tensor(sums)

    def set_totals(self, rho, sums):
        self.totals = (rho.clone(), sums.clone())

    def force(self, pos, q):
        t = np.arange(self.lo, self.hi)
        r = self.O.rbe(self.s, self.pos_all, self.q_all, self.k, mode=1, targets=t)
        return torch.as_tensor(r["force"])


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2405_06333_gb300.sharded import ShardedEvaluator
    from paper_2405_06333_gb300.synthetic import positions_charges
    s = O.System(Lx=12.0, Ly=10.0, H=3.0, Lz=40.0, gamma_top=0.5, gamma_bot=-0.7, alpha=0.9, M=5)
    N = 301
    pos, q = positions_charges(N, 12.0, 10.0, 3.0, seed=4)
    lo, hi = (0, 150) if rank == 0 else (150, N)
    be = OracleShardBackend(s, pos, q, lo, hi, P=40, seed=9)
    ev = ShardedEvaluator(be)
    F = ev.force(torch.as_tensor(pos[lo:hi]), torch.as_tensor(q[lo:hi]), step=2)
    rho_t, sums_t = be.totals
    k = O.sample_k(s, 9, 2, 40)
    ok_rho = np.allclose(rho_t.numpy(), O.rho_sigma(s, pos, q, k), rtol=0, atol=1e-10)
    ok_sum = np.allclose(sums_t.numpy(), [q.sum(), (q * q).sum(), np.sum(q * pos[:, 2]), np.abs(q).sum()],
                         rtol=0, atol=1e-10)
    full = O.rbe(s, pos, q, k, mode=1)["force"][lo:hi]
    ok_f = np.allclose(F.numpy(), full, rtol=1e-12, atol=1e-12)
    out[rank] = int(ok_rho) * 4 + int(ok_sum) * 2 + int(ok_f)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_two_rank_exchange_with_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert out[0] == 7 and out[1] == 7, dict(out)
