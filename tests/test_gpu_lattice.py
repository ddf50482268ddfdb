"""GPU parity of the deterministic lattice sum (rbe2d_force_lattice): the k-space sum of
Eq. 3.16 with the re-calibrated images of Sec. 3.4 over every k != 0 of a box, weighted
by w(k) = exp(-k^2/4alpha^2) (Eq. 2.21).

- against the oracle's sum over the same full lattice (its explicit k list and weights,
  both signs of every k): forces, energies and dU/dq, rel-L2 <= 1e-5 (FP64 mode) /
  1e-4 (FP32 mode), with several chunks and a ragged last chunk;
- plus the GPU real-space part, against the independent exact Ewald2D sum of the real
  and image charges (no L_z at all): the quasi-2D limit of Theorem 3.3;
- the random-batch mean over many steps approaches it (Theorem 2.3) on the same box.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import positions_charges
from tests import pin_ewald2d as E2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-5, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def model(Lx, Ly, H, n_max, P, gt, gb, M, alpha, precision, Lz=-1.0, r_c=-1.0, real_space=False):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    return RBE2D(Lx, Ly, H, n_max=n_max, P=P, gamma_top=gt, gamma_bot=gb, M=M, Lz=Lz, alpha=alpha, r_c=r_c,
                 precision=precision, real_space=real_space)


def osys(m, Lx, Ly, H, gt, gb):
    d = m.derived
    return O.System(Lx=Lx, Ly=Ly, H=H, Lz=d["Lz"], gamma_top=gt, gamma_bot=gb, alpha=d["alpha"], M=d["M"])


CASES = [
    # (Lx, Ly, H, N, gt, gb, M, alpha, nmax, P): dielectric, 12 chunks with a ragged last
    # one (1534 half-lattice entries, P = 128); homogeneous; one chunk larger than needed
    (10.0, 12.0, 3.0, 400, 0.7, -0.5, 6, 1.0, (4, 5, 15), 128),
    (9.0, 9.0, 4.0, 301, 0.0, 0.0, 0, 0.8, (3, 3, 9), 64),
    (8.0, 11.0, 2.0, 64, -0.9, 0.95, 9, 1.2, (2, 3, 6), 512),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_lattice_sum_matches_oracle(precision, case):
    Lx, Ly, H, N, gt, gb, M, a, nm, P = CASES[case]
    pos, q = positions_charges(N, Lx, Ly, H, seed=60 + case)
    m = model(Lx, Ly, H, N, P, gt, gb, M, a, precision)
    F, phi, e = m.force_lattice(dev(pos), dev(q), nm, energy=True, potential=True)
    torch.cuda.synchronize()
    s = osys(m, Lx, Ly, H, gt, gb)
    k, w = O.full_klist(s, list(nm))
    assert k.shape[0] == (2 * nm[0] + 1) * (2 * nm[1] + 1) * (2 * nm[2] + 1) - 1
    r = O.kspace(s, pos, q, k, w, mode=1, want_dq=True)
    eF = rel_l2(F.cpu().numpy(), r["force"])
    ePhi = rel_l2(phi.cpu().numpy(), r["dUdq"])
    print(f"case {case} {precision}: lattice force rel-L2 {eF:.2e}, dU/dq {ePhi:.2e}")
    assert eF < TOL[precision] and ePhi < TOL[precision]
    eg = e.cpu().numpy()
    for j in range(3):
        assert eg[j] == pytest.approx(r["energy"][j], rel=TOL[precision], abs=1e-12)
    assert eg[3] == 0.0
    m.close()


def test_lattice_sum_accumulates_and_is_deterministic():
    Lx, Ly, H, N, gt, gb, M, a, nm, P = CASES[0]
    pos, q = positions_charges(N, Lx, Ly, H, seed=60)
    m = model(Lx, Ly, H, N, P, gt, gb, M, a, "fp64")
    F1 = m.force_lattice(dev(pos), dev(q), nm)
    F2 = m.force_lattice(dev(pos), dev(q), nm)
    assert torch.equal(F1, F2)
    F3 = F1.clone()
    m.force_lattice(dev(pos), dev(q), nm, out=F3, accumulate=True)
    # the chunks now add onto F1 instead of onto zero: equal up to rounding
    assert rel_l2(F3.cpu().numpy(), 2 * F1.cpu().numpy()) < 1e-13
    m.close()


def test_lattice_sum_rejects_bad_arguments():
    m = model(10.0, 10.0, 2.0, 16, 32, 0.0, 0.0, 0, 1.0, "fp32")
    x = torch.zeros((16, 3), dtype=torch.float64, device="cuda")
    qv = torch.zeros(16, dtype=torch.float64, device="cuda")
    F = torch.empty((16, 3), device="cuda")
    for bad_nm, fl in (((0, 0, 0), 0), ((-1, 2, 2), 0), ((2, 2, 2), B.RBE2D_REAL), ((2, 2, 2), B.RBE2D_HOST_BUFFERS)):
        code = B.status_code(B.rbe2d_force_lattice, m.ctx, 16, x, qv, fl, bad_nm, F)
        assert code == B.RBE2D_EINVAL, (bad_nm, fl)
    m.close()


@pytest.mark.parametrize("gt,gb,M", [(0.0, 0.0, 0), (-0.7, 0.4, 5), (0.5, -0.8, 4)])
def test_lattice_plus_real_space_is_the_exact_quasi_2d_sum(gt, gb, M):
    """GPU lattice sum (L_z by Eq. 3.23 at eps = 1e-9, the whole Gaussian box) + GPU
    real space with images = the exact Ewald2D energy of the truncated image system."""
    Lx, Ly, H, a, r_c = 10.0, 12.0, 3.0, 1.0, 6.5
    rng = np.random.default_rng(9)
    N = 6
    pos = np.column_stack([rng.uniform(0, Lx, N), rng.uniform(0, Ly, N), rng.uniform(0.2, H - 0.2, N)])
    q = np.array([1.0, -1.0, 2.0, -2.0, 0.5, -0.5])
    Lz = O.auto_Lz(Lx, Ly, H, M, a, 1e-9)
    m = model(Lx, Ly, H, N, 4096, gt, gb, M, a, "fp64", Lz=Lz, r_c=r_c, real_space=True)
    nm = [O.nmax(a, L) for L in (Lx, Ly, m.derived["Lz"])]
    F, e = m.force_lattice(dev(pos), dev(q), nm, energy=True)
    Fr = torch.empty_like(F)
    er = torch.zeros(4, dtype=torch.float64, device="cuda")
    B.rbe2d_force(m.ctx, N, dev(pos), dev(q), B.RBE2D_REAL | B.RBE2D_ENERGY, Fr, None, er)
    torch.cuda.synchronize()
    U = float(e[:3].sum()) + float(er[3])
    Uex = E2.dielectric_energy(pos, q, Lx, Ly, H, gt, gb, M, a)
    assert U == pytest.approx(Uex, abs=2e-7 * np.sum(np.abs(q)))
    # forces against -grad of the exact energy (central differences)
    Ft = (F + Fr).cpu().numpy()
    h = 1e-5
    for i, d in ((0, 0), (2, 2), (5, 1)):
        p1, p2 = pos.copy(), pos.copy()
        p1[i, d] += h
        p2[i, d] -= h
        fd = -(E2.dielectric_energy(p1, q, Lx, Ly, H, gt, gb, M, a)
               - E2.dielectric_energy(p2, q, Lx, Ly, H, gt, gb, M, a)) / (2 * h)
        assert Ft[i, d] == pytest.approx(fd, abs=2e-6), (i, d)
    m.close()


def test_random_batch_mean_approaches_the_lattice_sum():
    """Theorem 2.3 on the GPU alone: over the sampler's own box, the mean of 600 batches
    of the random-batch force is within 5 standard errors of the lattice sum."""
    Lx, Ly, H, N, gt, gb, M, a = 8.0, 8.0, 2.0, 12, 0.7, -0.5, 4, 0.6
    pos, q = positions_charges(N, Lx, Ly, H, seed=13)
    m = model(Lx, Ly, H, N, 20, gt, gb, M, a, "fp64", Lz=24.0)
    nm = [O.nmax(a, L) for L in (Lx, Ly, 24.0)]
    Fs = []
    for step in range(600):
        m.sample_k(step)
        Fs.append(m.force(dev(pos), dev(q)).cpu().numpy())
    Fs = np.stack(Fs)
    ml = model(Lx, Ly, H, N, 1024, gt, gb, M, a, "fp64", Lz=24.0)
    Fl = ml.force_lattice(dev(pos), dev(q), nm).cpu().numpy()
    se = Fs.std(0, ddof=1) / np.sqrt(len(Fs))
    assert np.all(np.abs(Fs.mean(0) - Fl) < 5 * se + 1e-12)
    m.close()
    ml.close()


def test_force_variance_is_independent_of_Lz_and_scales_as_1_over_P():
    """The mean squared deviation of the random-batch force from the lattice sum (its
    variance) stays the same when the extended period L_z doubles and doubles again,
    and halves when P doubles (Sec. 2.3 and Sec. 3.3: S grows with V, the per-sample
    term does not)."""
    Lx, Ly, H, N, gt, gb, M, a = 10.0, 10.0, 3.0, 60, 0.6, -0.4, 6, 0.8
    pos, q = positions_charges(N, Lx, Ly, H, seed=31)
    X, Q = dev(pos), dev(q)
    R = 1000

    def mse(Lz, P):
        ml = model(Lx, Ly, H, N, 4096, gt, gb, M, a, "fp64", Lz=Lz)
        nm = [O.nmax(a, L) for L in (Lx, Ly, Lz)]
        Fl = ml.force_lattice(X, Q, nm)
        ml.close()
        m = model(Lx, Ly, H, N, P, gt, gb, M, a, "fp64", Lz=Lz)
        out = torch.empty((R, N, 3), dtype=torch.float64, device="cuda")
        for step in range(R):
            m.sample_k(step)
            m.force(X, Q, out=out[step])
        m.close()
        return float(((out - Fl) ** 2).sum(dim=(1, 2)).mean() / N)

    v = {Lz: mse(Lz, 16) for Lz in (30.0, 60.0, 120.0)}
    print("force variance vs Lz:", v)
    assert max(v.values()) / min(v.values()) < 1.3
    v32 = mse(60.0, 32)
    print("P = 32:", v32, "ratio", v[60.0] / v32)
    assert 1.6 < v[60.0] / v32 < 2.5


def test_force_variance_along_langevin_trajectories_is_independent_of_Lz():
    """The random-batch force variance on configurations of Langevin trajectories, not
    only on a fixed one.  Two NVT runs at the benchmark slab's density, contrasts and
    image count in a smaller cell (16 x 16 x 20, N = 6400, alpha = 1.0772, M = 14; WCA
    pairs and walls, dt = 5e-4, gamma = 10, kT = 1; a disordered start), one driven by the
    random-batch force at the L_z of Eq. 3.23 and one at twice it.  On six snapshots of
    each run (every 300 steps after 1500 steps of relaxation), the mean squared deviation of the random-batch k-space force (P = 100, 1000
    batches) from the lattice sum over the sampler's whole box -- the variance of
    Theorem 2.3 -- is taken at both L_z.  The variance follows the configuration (it falls
    as the start relaxes) and its estimate is heavy-tailed (rare wave vectors dominate
    it), so L_z is compared on the same snapshots with many batches: the mean ratio
    V(2 L_z) / V(L_z) is 1 within its standard error (Sec. 4.1: the variance does not
    grow with L_z)."""
    from paper_2405_06333_gb300.synthetic import random_positions_min_distance
    Lx, Ly, H, N, gt, gb, M, a = 16.0, 16.0, 20.0, 6400, 0.9, -0.9, 14, 1.0772173450159417
    pos0, q0 = random_positions_min_distance(N, Lx, Ly, H, 0.5, margin=0.25, seed=7)
    m0 = model(Lx, Ly, H, N, 100, gt, gb, M, a, "fp32")
    Lz0 = m0.derived["Lz"]  # Eq. 3.23 at eps = 1e-4
    m0.close()
    Lzs = (Lz0, 2.0 * Lz0)
    R, P, snaps, every, settle = 1000, 100, 6, 300, 1500
    flags = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL
    md = B.rbe2d_md_params(dt=5e-4, gamma=10.0, kT=1.0, mass=1.0, sigma_lj=0.5, eps_lj=1.0, sigma_wall=0.25,
                           eps_wall=1.0, noise_seed=9, force_flags=flags)
    evals = {Lz: (model(Lx, Ly, H, N, 4096, gt, gb, M, a, "fp32", Lz=Lz),
                  model(Lx, Ly, H, N, P, gt, gb, M, a, "fp32", Lz=Lz),
                  [O.nmax(a, L) for L in (Lx, Ly, Lz)]) for Lz in Lzs}
    buf = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    per = torch.empty(R, dtype=torch.float64, device="cuda")

    def variance(Lz, pos, q, salt):
        """Mean over R batches of sum_i |F_i - F_i^lattice|^2 / N, and its standard error."""
        ml, mr, nm = evals[Lz]
        Fl = ml.force_lattice(pos, q, nm).double()
        for r in range(R):
            mr.sample_k(salt + r)
            mr.force(pos, q, out=buf)
            per[r] = ((buf.double() - Fl) ** 2).sum()
        v = per.cpu().numpy() / N
        return v.mean(), v.std(ddof=1) / np.sqrt(R)

    report, ratios, own = [], [], {}
    for run_Lz in Lzs:
        st = torch.cuda.current_stream()
        p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=run_Lz, gamma_top=gt, gamma_bot=gb, M=M, alpha=a, r_c=-1, P=P,
                           seed=4, eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=1)
        ctx = B.rbe2d_init(p, N, st)
        pos = dev(pos0)
        vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
        q = dev(q0)
        F = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
        step = torch.zeros(1, dtype=torch.int64, device="cuda")
        B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, None)
        rows = []
        for _ in range(settle):  # the random start relaxes first (its variance falls by ~3x)
            B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, None)
        for snap in range(snaps):
            for _ in range(every):
                B.rbe2d_md_step(ctx, N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, None)
            (v1, e1), (v2, e2) = [variance(Lz, pos, q, 100000 * snap + 10000 * j) for j, Lz in enumerate(Lzs)]
            rows.append((v1, e1, v2, e2))
            ratios.append((v2 / v1, (v2 / v1) * np.hypot(e1 / v1, e2 / v2)))
        B.rbe2d_sync_status(ctx)
        B.rbe2d_destroy(ctx)
        assert torch.isfinite(pos).all()
        own[run_Lz] = [r[0] if run_Lz == Lz0 else r[2] for r in rows]
        report.append(f"run at Lz = {run_Lz:g}: " + ", ".join(f"{v1:.1f}+-{e1:.1f} / {v2:.1f}+-{e2:.1f}"
                                                             for v1, e1, v2, e2 in rows))
    for ml, mr, _ in evals.values():
        ml.close()
        mr.close()
    r = np.array([x for x, _ in ratios])
    se = np.array([e for _, e in ratios])
    w = 1.0 / se ** 2
    mean = float(np.sum(w * r) / np.sum(w))
    mean_se = float(1.0 / np.sqrt(np.sum(w)))
    print(f"force variance along NVT trajectories (V(Lz0) / V(2 Lz0) per snapshot): {'; '.join(report)}; "
          f"ratio V(2 Lz0)/V(Lz0) = {mean:.4f} +- {mean_se:.4f}; own-L_z means {own}")
    assert abs(mean - 1.0) < 4.0 * mean_se + 0.02
    assert abs(mean - 1.0) < 0.1
