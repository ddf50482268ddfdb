"""Particle-sharded evaluation emulated on one GPU: three shards, each with its own
context, exchange the partial structure factors and charge sums by a host-side sum; the
concatenated shard forces equal the unsharded forces."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2405_06333_gb300.synthetic import WORKLOADS, positions_charges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_three_shards_equal_the_whole(precision):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    from paper_2405_06333_gb300.sharded import CudaShardBackend
    w = WORKLOADS["dielectric_n1e4"]
    pos, q = positions_charges(w.N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    kw = dict(P=w.P, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M, Lz=w.Lz, alpha=w.alpha, seed=3,
              precision=precision)
    whole = RBE2D(w.Lx, w.Ly, w.H, n_max=w.N, **kw)
    whole.sample_k(5)
    F_ref = whole.force(torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")).cpu().numpy()
    cuts = [0, 3001, 7777, w.N]
    shards = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        m = RBE2D(w.Lx, w.Ly, w.H, n_max=b - a, **kw)
        shards.append((CudaShardBackend(m), torch.as_tensor(pos[a:b], device="cuda"),
                       torch.as_tensor(q[a:b], device="cuda"), m))
    parts = []
    for be, p_, q_, _ in shards:
        be.sample(5)
        parts.append(be.partial(p_, q_))
    rho = sum(r for r, _ in parts)
    sums = sum(s for _, s in parts)
    F = []
    for be, p_, q_, _ in shards:
        be.set_totals(rho, sums)
        F.append(be.force(p_, q_).cpu().numpy())
    F = np.concatenate(F)
    err = np.linalg.norm(F - F_ref) / np.linalg.norm(F_ref)
    assert err < (1e-12 if precision == "fp64" else 1e-5), err
    for *_, m in shards:
        m.close()
    whole.close()
