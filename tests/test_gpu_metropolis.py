"""GPU Metropolis variant of the k sampler: bit-exact chains against the oracle's chain
(integer states and acceptance counts), the downstream force on a Metropolis batch, and
the statistical comparison with the exact i.i.d. sampler that the variant exists for:
both estimators are unbiased for the lattice sum, the Metropolis batches are correlated
in time (the paper's Theorem 2.3 variance bound assumes independent batches)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import WORKLOADS, positions_charges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def model(Lx, Ly, H, n_max, P, gt, gb, M, alpha, Lz=-1.0, seed=0, precision="fp64"):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    return RBE2D(Lx, Ly, H, n_max=n_max, P=P, gamma_top=gt, gamma_bot=gb, M=M, Lz=Lz, alpha=alpha, seed=seed,
                 precision=precision)


def osys(m, Lx, Ly, H, gt, gb):
    d = m.derived
    return O.System(Lx=Lx, Ly=Ly, H=H, Lz=d["Lz"], gamma_top=gt, gamma_bot=gb, alpha=d["alpha"], M=d["M"])


GEOMS = [
    # (Lx, Ly, H, gt, gb, M, alpha, P, seed): a small dielectric cell; the 1e6-particle
    # slab's parameters (L = 200, Lz = 594, alpha = 1.077, P = 500)
    (20.0, 16.0, 4.0, 0.7, -0.5, 6, 0.9, 300, 5),
    ("slab_n1e6",),
]


def _geom(g):
    if g[0] == "slab_n1e6":
        w = WORKLOADS["slab_n1e6"]
        return (w.Lx, w.Ly, w.H, w.gamma_top, w.gamma_bot, w.M, w.alpha, w.P, w.seed, w.Lz)
    return tuple(g) + (-1.0,)


@pytest.mark.parametrize("g", range(len(GEOMS)))
def test_chains_match_the_oracle_bit_for_bit(g):
    Lx, Ly, H, gt, gb, M, a, P, seed, Lz = _geom(GEOMS[g])
    m = model(Lx, Ly, H, 8, P, gt, gb, M, a, Lz=Lz, seed=seed)
    s = osys(m, Lx, Ly, H, gt, gb)
    kout = torch.empty((P, 3), dtype=torch.int32, device="cuda")
    B.rbe2d_metropolis_reset(m.ctx, None)
    state = O.sample_k(s, seed, 0, P)  # the stationary start: the i.i.d. draw of step 0
    acc_o = 0
    for step, sweeps in ((1, 1), (2, 3), (3, 10), (7, 2)):
        B.rbe2d_sample_k_metropolis(m.ctx, step, sweeps, kout)
        state, a_ = O.metropolis(s, seed, step, sweeps, state)
        acc_o += a_
        assert np.array_equal(kout.cpu().numpy(), state), (step, sweeps)
    assert B.rbe2d_metropolis_accepted(m.ctx) == acc_o
    # explicit cold start
    start = np.tile(np.array([1, 0, 0], np.int32), (P, 1))
    B.rbe2d_metropolis_reset(m.ctx, dev(start, torch.int32))
    B.rbe2d_sample_k_metropolis(m.ctx, 4, 5, kout)
    st2, a2 = O.metropolis(s, seed, 4, 5, start)
    assert np.array_equal(kout.cpu().numpy(), st2)
    assert B.rbe2d_metropolis_accepted(m.ctx) == a2
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_force_on_a_metropolis_batch_matches_the_oracle(precision):
    Lx, Ly, H, gt, gb, M, a, P, seed = 20.0, 16.0, 4.0, 0.7, -0.5, 6, 0.9, 300, 5
    N = 3000
    pos, q = positions_charges(N, Lx, Ly, H, seed=21)
    m = model(Lx, Ly, H, N, P, gt, gb, M, a, seed=seed, precision=precision)
    kout = torch.empty((P, 3), dtype=torch.int32, device="cuda")
    B.rbe2d_metropolis_reset(m.ctx, None)
    B.rbe2d_sample_k_metropolis(m.ctx, 1, 4, kout)
    F = m.force(dev(pos), dev(q))
    s = osys(m, Lx, Ly, H, gt, gb)
    Fo = O.rbe(s, pos, q, kout.cpu().numpy(), mode=1)["force"]
    assert rel_l2(F.cpu().numpy(), Fo) < (1e-5 if precision == "fp64" else 1e-4)
    m.close()


def test_metropolis_and_exact_sampler_statistics():
    """Both estimators average to the lattice sum (batch means over blocks of 25 steps,
    5 standard errors); the i.i.d. batches are uncorrelated from step to step while the
    one-update Metropolis batches are strongly correlated (lag-1 autocorrelation of the
    force on one particle), which more updates per step reduce."""
    Lx, Ly, H, N, gt, gb, M, a = 8.0, 8.0, 2.0, 12, 0.7, -0.5, 4, 0.6
    pos, q = positions_charges(N, Lx, Ly, H, seed=13)
    P, R = 20, 2000
    X, Q = dev(pos), dev(q)
    nm = [O.nmax(a, L) for L in (Lx, Ly, 24.0)]
    ml = model(Lx, Ly, H, N, 1024, gt, gb, M, a, Lz=24.0)
    Fl = ml.force_lattice(X, Q, nm).cpu().numpy()
    ml.close()

    def run(kind, sweeps=1):
        m = model(Lx, Ly, H, N, P, gt, gb, M, a, Lz=24.0, seed=17)
        if kind == "mh":
            B.rbe2d_metropolis_reset(m.ctx, None)
        out = torch.empty((R, N, 3), dtype=torch.float64, device="cuda")
        for step in range(R):
            if kind == "mh":
                B.rbe2d_sample_k_metropolis(m.ctx, step + 1, sweeps, None)
            else:
                m.sample_k(step)
            m.force(X, Q, out=out[step])
        acc = B.rbe2d_metropolis_accepted(m.ctx) / (R * P * sweeps) if kind == "mh" else None
        m.close()
        return out.cpu().numpy(), acc

    def lag1(x):
        x = x - x.mean()
        return float(np.dot(x[:-1], x[1:]) / np.dot(x, x))

    stats = {}
    for kind, sweeps in (("iid", 1), ("mh", 1), ("mh", 10)):
        Fs, acc = run(kind, sweeps)
        blocks = Fs.reshape(R // 25, 25, N, 3).mean(1)
        se = blocks.std(0, ddof=1) / np.sqrt(blocks.shape[0])
        z = np.abs(Fs.mean(0) - Fl) / (se + 1e-300)
        rho = np.mean([lag1(Fs[:, i, d]) for i in range(N) for d in range(3)])
        stats[(kind, sweeps)] = (float(z.max()), rho, float(Fs.var(0).mean()), acc)
        print(kind, sweeps, "max z", z.max(), "mean lag-1 autocorrelation", rho, "acceptance", acc)
        assert z.max() < 5.0
    assert abs(stats[("iid", 1)][1]) < 0.1
    assert stats[("mh", 1)][1] > 0.3
    assert stats[("mh", 10)][1] < stats[("mh", 1)][1]
    # per-step variance is the same distribution's: within 25 % of the i.i.d. one
    v0 = stats[("iid", 1)][2]
    for key in (("mh", 1), ("mh", 10)):
        assert abs(stats[key][2] / v0 - 1.0) < 0.25
