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
            kc=1.0, skin=0.0):
    p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=-1, gamma_top=gt, gamma_bot=gb, M=M, alpha=alpha, r_c=-1, P=P, seed=5,
                       eps=1e-4, precision=precision, coulomb_k=kc, real_space=real, skin=skin)
    return B.rbe2d_init(p, N, stream)


def mdp(flags, sigma_lj=0.5, sigma_wall=0.25, dt=0.002, gamma=1.0, kT=1.0, seed=11):
    return B.rbe2d_md_params(dt=dt, gamma=gamma, kT=kT, mass=1.0, sigma_lj=sigma_lj, eps_lj=1.0,
                             sigma_wall=sigma_wall, eps_wall=1.0, noise_seed=seed, force_flags=flags)


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_graph_replay_equals_eager_bitwise(skin):
    Lx, Ly, H, N = 16.0, 16.0, 4.0, 1200
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=3)
    s = torch.cuda.Stream()
    flags = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL
    md = mdp(flags)
    results = []
    for use_graph in (False, True):
        ctx = ctx_for(Lx, Ly, H, N, s, skin=skin)
        assert B.rbe2d_md_list_stats(ctx)["enabled"] == (skin > 0)
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


def test_resume_from_a_checkpoint_is_bitwise():
    """Checkpoint and resume: the MD state is the positions, the velocities, the last force
    and the step counter; the batch and the thermostat noise come from counter-based Philox
    keyed by the step, so no generator state is saved.  Ten steps, a checkpoint copied to
    the host, a fresh context restored from it and ten more steps give the same bits as
    twenty steps without a break (cell-scan real space, which depends on the positions
    alone)."""
    Lx, Ly, H, N = 16.0, 16.0, 4.0, 1200
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=4)
    s = torch.cuda.Stream()
    md = mdp(B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL)

    def start(state=None):
        ctx = ctx_for(Lx, Ly, H, N, s)
        with torch.cuda.stream(s):
            if state is None:
                t = {"pos": torch.as_tensor(pos0, device="cuda").contiguous(),
                     "vel": torch.zeros((N, 3), dtype=torch.float64, device="cuda"),
                     "F": torch.zeros((N, 3), dtype=torch.float32, device="cuda"),
                     "step": torch.zeros(1, dtype=torch.int64, device="cuda")}
            else:
                t = {k: torch.as_tensor(v, device="cuda").contiguous() for k, v in state.items()}
            q = torch.as_tensor(q0, device="cuda")
        s.synchronize()
        if state is None:
            B.rbe2d_md_step(ctx, N, t["pos"], t["vel"], q, t["F"], t["step"], md, B.RBE2D_MD_FORCE, None)
        return ctx, t, q

    def run(ctx, t, q, n):
        for _ in range(n):
            B.rbe2d_md_step(ctx, N, t["pos"], t["vel"], q, t["F"], t["step"], md, B.RBE2D_MD_STEP, None)
        s.synchronize()
        B.rbe2d_sync_status(ctx)

    ctx, t, q = start()
    run(ctx, t, q, 20)
    whole = {k: v.cpu().numpy() for k, v in t.items()}
    B.rbe2d_destroy(ctx)

    ctx, t, q = start()
    run(ctx, t, q, 10)
    checkpoint = {k: v.cpu().numpy().copy() for k, v in t.items()}
    B.rbe2d_destroy(ctx)
    assert int(checkpoint["step"][0]) == 10
    ctx, t, q = start(checkpoint)
    run(ctx, t, q, 10)
    resumed = {k: v.cpu().numpy() for k, v in t.items()}
    B.rbe2d_destroy(ctx)

    assert int(resumed["step"][0]) == int(whole["step"][0]) == 20
    for k in ("pos", "vel", "F"):
        assert np.array_equal(resumed[k], whole[k]), k
    assert not np.array_equal(whole["pos"], pos0)


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


# ---------------------------------------------------------------- against the host reference
def _md_run(ctx, N, pos0, vel0, q0, md, step0, precision_dtype):
    """MD_FORCE at pos0, then one MD_STEP: returns (F0, pos, vel, F1, step) on the host."""
    pos = torch.as_tensor(pos0, device="cuda").contiguous().clone()
    vel = torch.as_tensor(vel0, device="cuda").contiguous().clone()
    q = torch.as_tensor(q0, device="cuda")
    F = torch.zeros((N, 3), dtype=precision_dtype, device="cuda")
    step = torch.full((1,), step0, dtype=torch.int64, device="cuda")
    B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, None)
    torch.cuda.synchronize()
    F0 = F.double().cpu().numpy()
    B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, None)
    torch.cuda.synchronize()
    B.rbe2d_sync_status(ctx)
    return F0, pos.cpu().numpy(), vel.cpu().numpy(), F.double().cpu().numpy(), int(step.item())


def _minimum_image(d, Lx, Ly):
    d = d.copy()
    d[:, 0] -= Lx * np.round(d[:, 0] / Lx)
    d[:, 1] -= Ly * np.round(d[:, 1] / Ly)
    return d


def test_positions_at_the_edges_stay_put_and_in_range():
    """No force, no friction, kT = 0 and no walls: a step leaves every position as it was,
    including the last double below Lx and Ly (where x L^-1 rounds to 1), 0 and -0.0 in
    x, y, and z exactly at 0 and H; every coordinate stays in [0, L) and [0, H]."""
    Lx, Ly, H, N = 12.0, 10.0, 4.0, 64
    rng = np.random.default_rng(4)
    pos0 = np.stack([rng.uniform(0, Lx, N), rng.uniform(0, Ly, N), rng.uniform(0, H, N)], axis=1)
    pos0[0] = [np.nextafter(Lx, 0.0), np.nextafter(Ly, 0.0), H]
    pos0[1] = [0.0, 0.0, 0.0]
    pos0[2] = [-0.0, -0.0, np.nextafter(H, 0.0)]
    pos0[3] = [Lx * (1 - 2.0 ** -52), Ly * (1 - 2.0 ** -52), 5e-324]
    q0 = np.zeros(N)
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, real=0, gt=0.0, gb=0.0, M=0)
    md = B.rbe2d_md_params(dt=1e-3, gamma=0.0, kT=0.0, mass=1.0, sigma_lj=0.0, eps_lj=0.0, sigma_wall=0.0,
                           eps_wall=0.0, noise_seed=2, force_flags=B.RBE2D_KSPACE)
    _, pos, vel, _, st = _md_run(ctx, N, pos0, np.zeros((N, 3)), q0, md, 0, torch.float32)
    B.rbe2d_destroy(ctx)
    assert st == 1 and np.all(vel == 0)
    assert np.array_equal(pos, pos0)  # -0.0 == 0.0
    assert np.all((pos[:, 0] >= 0) & (pos[:, 0] < Lx) & (pos[:, 1] >= 0) & (pos[:, 1] < Ly))
    assert np.all((pos[:, 2] >= 0) & (pos[:, 2] <= H))


def test_baoab_step_matches_host_reference():
    """One BAOAB step with kT = 0 (the O step is then v <- exp(-gamma dt) v exactly), the
    k-space + IBC force in float64 mode and the WCA walls, against tests/md_reference.py
    fed the force before the step and the force the library computed after it.  Particles
    sit inside both walls' range and move across the x and y cell edges."""
    from tests import md_reference as R
    Lx, Ly, H, N = 12.0, 10.0, 4.0, 2000
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=8)
    rng = np.random.default_rng(8)
    vel0 = rng.normal(0.0, 1.0, (N, 3))
    pos0[:6, 2] = [0.14, 0.2, 0.27, H - 0.15, H - 0.21, H - 0.26]        # within 2^(1/6) sigma of a wall
    pos0[6:10, 0] = [Lx - 1e-4, 1e-4, 5.0, 6.0]; pos0[8:10, 1] = [Ly - 1e-4, 1e-4]
    vel0[6:10, :2] = [[30.0, 0.0], [-30.0, 0.0], [0.0, 30.0], [0.0, -30.0]]  # across the cell edges
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, precision=B.RBE2D_FP64, real=0)
    dt, gamma, sw, ew = 0.002, 3.0, 0.25, 1.3
    md = B.rbe2d_md_params(dt=dt, gamma=gamma, kT=0.0, mass=1.7, sigma_lj=0.0, eps_lj=0.0, sigma_wall=sw,
                           eps_wall=ew, noise_seed=5, force_flags=B.RBE2D_KSPACE | B.RBE2D_IBC)
    F0, pos, vel, F1, st = _md_run(ctx, N, pos0, vel0, q0, md, 4, torch.float64)
    B.rbe2d_destroy(ctx)
    assert st == 5
    assert np.abs(F0).max() > 0.1 and np.abs(F1).max() > 0.1  # a real force drives the step
    xr, vr = R.baoab_step(pos0, vel0, F0, F1, dt=dt, gamma=gamma, kT=0.0, mass=1.7, H=H, Lx=Lx, Ly=Ly,
                          sigma_wall=sw, eps_wall=ew)
    assert np.abs(_minimum_image(pos - xr, Lx, Ly)).max() < 1e-12
    assert np.all((pos[:, 0] >= 0) & (pos[:, 0] < Lx) & (pos[:, 1] >= 0) & (pos[:, 1] < Ly))
    np.testing.assert_allclose(vel, vr, rtol=1e-12, atol=1e-12)
    # the wrapped particles really crossed an edge
    assert pos[6, 0] < 1.0 and pos[7, 0] > Lx - 1.0 and pos[8, 1] < 1.0 and pos[9, 1] > Ly - 1.0


@pytest.mark.parametrize("precision", [B.RBE2D_FP64, B.RBE2D_FP32_MIXED])
def test_wall_force_matches_closed_form(precision):
    """Particles at rest near z = 0 and z = H, no other force, no friction, kT = 0: one
    step gives v = (dt/2m)(F_w(z) + F_w(z')), z' the height the step reaches, as the BAOAB
    reference computes it with the closed-form WCA wall.  In the float32 mode the wall
    force is evaluated in float32 at z rounded to float32 (the distance d then carries an
    error of ~1e-7 H, and F ~ d^-13 amplifies it): rtol 1e-4 there."""
    from tests import md_reference as R
    Lx, Ly, H = 6.0, 6.0, 3.0
    z = np.array([0.1, 0.13, 0.16, 0.2, 0.24, 0.27, 0.3, H - 0.13, H - 0.18, H - 0.22, H - 0.27, H - 0.4])
    N = len(z)
    pos0 = np.stack([np.linspace(0.5, 5.5, N), np.linspace(5.5, 0.5, N), z], axis=1)
    q0 = np.zeros(N)
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, precision=precision, real=0, gt=0.0, gb=0.0, M=0)
    dt, sw, ew, m = 1e-3, 0.25, 1.3, 2.0
    md = B.rbe2d_md_params(dt=dt, gamma=0.0, kT=0.0, mass=m, sigma_lj=0.0, eps_lj=0.0, sigma_wall=sw, eps_wall=ew,
                           noise_seed=1, force_flags=0)
    dtype = torch.float64 if precision == B.RBE2D_FP64 else torch.float32
    F0, pos, vel, F1, _ = _md_run(ctx, N, pos0, np.zeros((N, 3)), q0, md, 0, dtype)
    B.rbe2d_destroy(ctx)
    assert np.all(F0 == 0) and np.all(F1 == 0)
    xr, vr = R.baoab_step(pos0, np.zeros((N, 3)), F0, F1, dt=dt, gamma=0.0, kT=0.0, mass=m, H=H, Lx=Lx, Ly=Ly,
                          sigma_wall=sw, eps_wall=ew)
    rtol = 1e-12 if precision == B.RBE2D_FP64 else 1e-4
    np.testing.assert_allclose(vel[:, 2], vr[:, 2], rtol=rtol, atol=1e-300)
    np.testing.assert_allclose(pos[:, 2] - z, xr[:, 2] - z, rtol=rtol, atol=1e-15)
    assert np.all(vel[:, :2] == 0)
    # signs and range: pushed up near z = 0, down near z = H, nothing beyond 2^(1/6) sigma
    assert np.all(vel[:6, 2] > 0) and np.all(vel[7:11, 2] < 0) and vel[6, 2] == 0 and vel[11, 2] == 0


def test_thermostat_noise_matches_host_philox():
    """No force, no walls: one step gives v = c1 v0 + sqrt(1 - c1^2) sqrt(kT/m) xi with xi
    regenerated on the host from Philox4x32-10 (counter = particle, step; key = seed)."""
    from tests import md_reference as R
    Lx, Ly, H, N = 10.0, 10.0, 5.0, 5000
    rng = np.random.default_rng(3)
    pos0 = np.stack([rng.uniform(0, Lx, N), rng.uniform(0, Ly, N), rng.uniform(1.0, H - 1.0, N)], axis=1)
    vel0 = rng.normal(0.0, 0.5, (N, 3))
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, precision=B.RBE2D_FP64, real=0, gt=0.0, gb=0.0, M=0)
    seed, step0 = 0x1234_5678_9ABC, 5
    dt, gamma, kT, m = 0.01, 2.0, 1.7, 1.3
    md = B.rbe2d_md_params(dt=dt, gamma=gamma, kT=kT, mass=m, sigma_lj=0.0, eps_lj=0.0, sigma_wall=0.0,
                           eps_wall=0.0, noise_seed=seed, force_flags=0)
    F0, pos, vel, F1, st = _md_run(ctx, N, pos0, vel0, np.zeros(N), md, step0, torch.float64)
    B.rbe2d_destroy(ctx)
    assert st == step0 + 1
    xi = R.thermostat_normals(N, step0, seed)
    xr, vr = R.baoab_step(pos0, vel0, F0, F1, dt=dt, gamma=gamma, kT=kT, mass=m, H=H, Lx=Lx, Ly=Ly, xi=xi)
    c1 = np.exp(-gamma * dt)
    noise = np.sqrt(1 - c1 * c1) * np.sqrt(kT / m) * xi
    # the normals are made in float32 on the device: a few float32 ulps of the noise term
    assert np.all(np.abs(vel - vr) <= 4e-6 * np.abs(noise) + 1e-12)
    assert np.abs(_minimum_image(pos - xr, Lx, Ly)).max() < 1e-7


def test_pair_lists_match_the_cell_scan_along_a_trajectory():
    """The MD step's real-space and WCA force through the pair lists (skin 0.3, rebuilt on
    the device when a charge has moved more than skin / 2) equals the cell scan's at the
    same positions, up to float32 summation order, at the start and along a trajectory
    that needs several rebuilds; a change of N forces a rebuild too."""
    Lx, Ly, H, N = 24.0, 24.0, 8.0, 6000
    pos0, q0 = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=12)
    s = torch.cuda.current_stream()
    flags = B.RBE2D_REAL
    md = mdp(flags, sigma_lj=0.5, dt=0.004, gamma=1.0, kT=1.0, seed=21)
    ctx_l = ctx_for(Lx, Ly, H, N, s, skin=0.3)
    ctx_c = ctx_for(Lx, Ly, H, N, s, skin=0.0)
    assert B.rbe2d_md_list_stats(ctx_l)["enabled"] and not B.rbe2d_md_list_stats(ctx_c)["enabled"]
    pos = torch.as_tensor(pos0, device="cuda").contiguous()
    vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    q = torch.as_tensor(q0, device="cuda")
    F = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")

    def cell_force(p):
        Fc = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
        B.rbe2d_md_step(ctx_c, N, p.clone(), torch.zeros_like(vel), q, Fc, torch.zeros_like(step), md,
                        B.RBE2D_MD_FORCE, None)
        return Fc

    def rel(a, b):
        return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))

    B.rbe2d_md_step(ctx_l, N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, None)
    errs = [rel(F, cell_force(pos))]
    for _ in range(6):
        for _ in range(25):
            B.rbe2d_md_step(ctx_l, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, None)
        errs.append(rel(F, cell_force(pos)))
    B.rbe2d_sync_status(ctx_l)
    B.rbe2d_sync_status(ctx_c)
    builds = B.rbe2d_md_list_stats(ctx_l)["builds"]
    print(f"pair lists vs cell scan: rel-L2 {[f'{e:.1e}' for e in errs]}, {builds} builds in 150 steps")
    assert max(errs) < 1e-5
    assert 2 <= builds < 150  # rebuilt when needed, not every step
    # a smaller N (the first N / 2 charges) rebuilds and still matches
    n2 = N // 2
    p2, q2 = pos[:n2].contiguous(), q[:n2].contiguous()
    F2 = torch.zeros((n2, 3), dtype=torch.float32, device="cuda")
    B.rbe2d_md_step(ctx_l, n2, p2, torch.zeros((n2, 3), dtype=torch.float64, device="cuda"), q2, F2,
                    torch.zeros_like(step), md, B.RBE2D_MD_FORCE, None)
    Fc2 = torch.zeros((n2, 3), dtype=torch.float32, device="cuda")
    B.rbe2d_md_step(ctx_c, n2, p2.clone(), torch.zeros((n2, 3), dtype=torch.float64, device="cuda"), q2, Fc2,
                    torch.zeros_like(step), md, B.RBE2D_MD_FORCE, None)
    assert rel(F2, Fc2) < 1e-5
    assert B.rbe2d_md_list_stats(ctx_l)["builds"] == builds + 1
    B.rbe2d_destroy(ctx_l)
    B.rbe2d_destroy(ctx_c)


def test_pair_list_capacity_overflow_is_reported():
    """A configuration far denser than the context's n_max / volume (every charge inside a
    4 x 4 x 3 corner of a 20 x 20 x 5 cell) gives lists longer than their capacity: the
    entries past it are dropped inside the kernel's bounds and rbe2d_sync_status reports
    RBE2D_ERANGE; a later configuration of normal density builds and evaluates cleanly."""
    Lx, Ly, H, N = 20.0, 20.0, 5.0, 2000
    s = torch.cuda.current_stream()
    ctx = ctx_for(Lx, Ly, H, N, s, skin=0.3, alpha=1.0)
    rng = np.random.default_rng(4)
    dense = np.stack([rng.uniform(0.5, 4.5, N), rng.uniform(0.5, 4.5, N), rng.uniform(1.0, 4.0, N)], axis=1)
    q = np.ones(N); q[N // 2:] = -1.0
    md = mdp(B.RBE2D_REAL, sigma_lj=0.0)
    F = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    qd = torch.as_tensor(q, device="cuda")
    B.rbe2d_md_step(ctx, N, torch.as_tensor(dense, device="cuda"), torch.zeros((N, 3), dtype=torch.float64,
                    device="cuda"), qd, F, step, md, B.RBE2D_MD_FORCE, None)
    with pytest.raises(B.RBE2DError) as ei:
        B.rbe2d_sync_status(ctx)
    assert ei.value.code == B.RBE2D_ERANGE
    pos, _ = lattice_positions_charges(N, Lx, Ly, H, margin=0.3, seed=2)
    B.rbe2d_md_step(ctx, N, torch.as_tensor(pos, device="cuda"), torch.zeros((N, 3), dtype=torch.float64,
                    device="cuda"), qd, F, step, md, B.RBE2D_MD_FORCE, None)
    B.rbe2d_sync_status(ctx)  # no error: the lists were rebuilt within their capacity
    assert torch.isfinite(F).all()
    B.rbe2d_destroy(ctx)
