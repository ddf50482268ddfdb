"""Langevin MD step (Eq. 2.27, BAOAB) with the RBE2D force: CUDA-graph replay equals
eager execution bit for bit, the thermostat holds kT, the force-only mode equals
rbe2d_force on the same batch, and the WCA pair force matches a brute-force sum."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import lattice_positions_charges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


def ctx_for(Lx, Ly, H, N, stream, precision=B.RBE2D_FP32_MIXED, gt=0.6, gb=-0.5, M=-1, P=64, real=1, alpha=1.2,
            kc=1.0):
    p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=-1, gamma_top=gt, gamma_bot=gb, M=M, alpha=alpha, r_c=-1, P=P, seed=5,
                       eps=1e-4, precision=precision, coulomb_k=kc, real_space=real)
    return B.rbe2d_init(p, N, stream)


def mdp(flags, sigma_lj=0.5, sigma_wall=0.25, dt=0.002, gamma=1.0, kT=1.0, seed=11):
    return B.rbe2d_md_params(dt=dt, gamma=gamma, kT=kT, mass=1.0, sigma_lj=sigma_lj, eps_lj=1.0,
                             sigma_wall=sigma_wall, eps_wall=1.0, noise_seed=seed, force_flags=flags)


def test_graph_replay_equals_eager_bitwise():
    Lx, Ly, H, N = 16.0, 16.0, 4.0, 1200
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=3)
    s = torch.cuda.Stream()
    flags = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL
    md = mdp(flags)
    results = []
    for use_graph in (False, True):
        ctx = ctx_for(Lx, Ly, H, N, s)
        with torch.cuda.stream(s):
            pos = torch.as_tensor(pos0, device="cuda").contiguous()
            vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
            q = torch.as_tensor(q0, device="cuda")
            F = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
            step = torch.zeros(1, dtype=torch.int64, device="cuda")
            stats = torch.zeros(2, dtype=torch.float64, device="cuda")
        B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, stats)
        if use_graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, stats)
            for _ in range(25):
                g.replay()
        else:
            for _ in range(25):
                B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, stats)
        s.synchronize()
        B.rbe2d_sync_status(ctx)
        results.append((pos.cpu().numpy(), vel.cpu().numpy(), int(step.item())))
        B.rbe2d_destroy(ctx)
    (pe, ve, se), (pg, vg, sg) = results
    assert se == 25 and sg == 25
    assert np.array_equal(pe, pg) and np.array_equal(ve, vg)
    assert np.all(np.isfinite(pe)) and pe[:, 2].min() >= 0 and pe[:, 2].max() <= H


def test_thermostat_reaches_kT():
    """Ideal particles between walls: the kinetic temperature 2 KE / (3 N) relaxes to kT."""
    Lx, Ly, H, N = 30.0, 30.0, 6.0, 20000
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=4)
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, real=0)
    md = mdp(0, sigma_lj=0.0, kT=1.7, gamma=5.0, dt=0.01)
    pos = torch.as_tensor(pos0, device="cuda").contiguous()
    vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    q = torch.as_tensor(q0, device="cuda")
    F = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, stats)
    temps = []
    for i in range(300):
        B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, stats)
        if i >= 100:
            temps.append(2.0 * float(stats[0]) / (3 * N))
    assert np.mean(temps) == pytest.approx(1.7, rel=0.02)
    B.rbe2d_destroy(ctx)


def test_force_mode_equals_rbe2d_force_on_the_same_batch():
    Lx, Ly, H, N = 20.0, 20.0, 5.0, 3000
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=5)
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s)
    flags = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL
    md = mdp(flags, sigma_lj=0.0)
    pos = torch.as_tensor(pos0, device="cuda").contiguous()
    vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    q = torch.as_tensor(q0, device="cuda")
    F = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    step = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, None)
    F2 = torch.empty_like(F)
    B.rbe2d_sample_k(ctx, 7, None)
    B.rbe2d_force(ctx, N, pos, q, flags, F2)
    torch.cuda.synchronize()
    assert torch.equal(F, F2)
    B.rbe2d_destroy(ctx)


def test_wca_pair_force_matches_brute_force():
    Lx, Ly, H, N = 8.0, 8.0, 3.0, 400
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=6, jitter=0.3)
    sig = 0.45
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, precision=B.RBE2D_FP64, real=1)
    pos = torch.as_tensor(pos0, device="cuda").contiguous()
    vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    q = torch.as_tensor(q0, device="cuda")
    F_lj = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.rbe2d_md_step(ctx, N, pos, vel, q, F_lj, step, mdp(0, sigma_lj=sig), B.RBE2D_MD_FORCE, None)
    torch.cuda.synchronize()
    # brute force, minimum image in x and y
    d = pos0[:, None, :] - pos0[None, :, :]
    d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
    d[..., 1] -= Ly * np.round(d[..., 1] / Ly)
    r2 = np.sum(d * d, axis=-1)
    np.fill_diagonal(r2, np.inf)
    mask = r2 < (2 ** (1 / 6) * sig) ** 2
    s6 = np.where(mask, (sig * sig / r2) ** 3, 0.0)
    f = np.where(mask, 24.0 * (2 * s6 * s6 - s6) / r2, 0.0)
    ref = np.sum(f[..., None] * d, axis=1)
    assert mask.sum() > 20
    np.testing.assert_allclose(F_lj.cpu().numpy(), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    B.rbe2d_destroy(ctx)
