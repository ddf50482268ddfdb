"""GPU parity of the k-space path (sample, structure factor, fold, force, adjoint)
against the FP64 CPU oracle, through the C ABI.

Bars (written here, from the build's target): relative L2 error over all compared
force components <= 1e-5 in RBE2D_FP64 mode and <= 1e-4 in RBE2D_FP32_MIXED mode; the
sampled wave-vector indices are integers and must match bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import WORKLOADS, positions_charges, random_kbatch

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


def make(w, precision, P=None, seed=None, n_max=None, **over):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    kw = dict(n_max=n_max or w.N, P=P or w.P, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M, Lz=w.Lz,
              alpha=w.alpha, r_c=w.r_c, seed=w.seed if seed is None else seed, precision=precision)
    kw.update(over)
    return RBE2D(w.Lx, w.Ly, w.H, **kw)


def osys(model, w):
    d = model.derived
    return O.System(Lx=w.Lx, Ly=w.Ly, H=w.H, Lz=d["Lz"], gamma_top=w.gamma_top, gamma_bot=w.gamma_bot,
                    alpha=d["alpha"], M=d["M"])


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


SMALL = ["plain_n1e3", "dielectric_n1e4"]


# ------------------------------------------------------------------ sampler
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_sampled_batch_matches_oracle_sampler(name):
    w = WORKLOADS[name]
    m = make(w, "fp32", n_max=16)
    s = osys(m, w)
    for step in (0, 1, 12345):
        k = m.sample_k(step, return_k=True).cpu().numpy()
        ko = O.sample_k(s, w.seed, step, w.P)
        assert np.array_equal(k, ko), (name, step)
    assert m.derived["S"] == pytest.approx(O.S(s), rel=1e-14)
    m.sync_status()
    m.close()


def test_sampler_matches_oracle_over_many_steps():
    """100,000 draws (200 steps of P = 500) at the benchmark slab, bit for bit: about 600
    of the 300,000 table searches start in the first or last guide bucket, whose bracket
    spans the flat tail of the Gaussian (hundreds of entries), so the cooperative search's
    long paths are exercised as well as the short ones."""
    w = WORKLOADS["slab_n1e6"]
    m = make(w, "fp32", n_max=16)
    s = osys(m, w)
    for step in range(1000, 1200):
        k = m.sample_k(step, return_k=True).cpu().numpy()
        ko = O.sample_k(s, w.seed, step, w.P)
        assert np.array_equal(k, ko), step
    m.sync_status()
    m.close()


# ------------------------------------------------------------------ structure factors
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1, 2, 511, 1000, 4097, 20011])
def test_structure_factors_match_oracle(precision, N):
    w = WORKLOADS["dielectric_n1e4"]
    pos, q = positions_charges(N, w.Lx, w.Ly, w.H, seed=5)
    if N % 2 == 1:
        q[-1] = 1.0  # the synthetic mix leaves an odd particle uncharged; give it a charge
    assert np.all(q != 0.0)
    m = make(w, precision, n_max=max(N, 1))
    s = osys(m, w)
    k = m.sample_k(3, return_k=True).cpu().numpy()
    rs = m.structure_factor(dev(pos), dev(q)).cpu().numpy()
    ref = O.rho_sigma(s, pos, q, k)
    # per-term error budget: FP32 mode rounds each phase (fixed-point quantisation
    # <= 1e-7 rad, int -> float <= 2e-7 rad) and each MUFU sin/cos (~4e-7): <= 1e-6 per
    # term, so |d rho| <= 1e-6 sum|q|; FP64 mode: <= 1e-13 per term.
    l1 = np.sum(np.abs(q)) + 1e-300
    err = np.abs(rs - ref).max() / l1
    print(f"N={N} {precision}: max|d rho|/sum|q| = {err:.3e}, /sqrt(sum q^2) = {err * l1 / np.sqrt(np.sum(q * q)):.3e}")
    assert err < (1e-13 if precision == "fp64" else 1e-6), err
    m.close()


@pytest.mark.parametrize("P", [33, 100, 200, 300, 400, 700])
def test_structure_factor_wave_vector_groups_at_every_batch_size(P):
    """Batch sizes whose k slots (k chunks x threads x wave vectors per thread) leave
    whole warp groups of 32 empty run the variant that skips them (P = 33, 200, 300,
    400, 700 at 4 wave vectors per thread; P = 100 fills its slots): every structure
    factor shape and both input precisions meet the same per-term bound against the
    oracle."""
    w = WORKLOADS["dielectric_n1e4"]
    N = 20011
    pos, q = positions_charges(N, w.Lx, w.Ly, w.H, seed=7)
    q[-1] = 1.0
    m = make(w, "fp32", P=P, n_max=N)
    s = osys(m, w)
    k = m.sample_k(1, return_k=True).cpu().numpy()
    # float32 inputs: the oracle takes the same rounded positions and charges
    pos32, q32 = pos.astype(np.float32).astype(np.float64), q.astype(np.float32).astype(np.float64)
    ref = {torch.float64: O.rho_sigma(s, pos, q, k), torch.float32: O.rho_sigma(s, pos32, q32, k)}
    l1 = np.sum(np.abs(q))
    for shape in (0, 1, 2):
        B.rbe2d_set_tuning(m.ctx, 2, 1, shape, 4)
        for dt in (torch.float64, torch.float32):
            rs = m.structure_factor(dev(pos, dt), dev(q, dt)).cpu().numpy()
            err = np.abs(rs - ref[dt]).max() / l1
            print(f"P={P} shape {shape} {dt}: max|d rho|/sum|q| = {err:.3e}")
            assert err < 1e-6, (P, shape, dt, err)
    m.close()


# ------------------------------------------------------------------ forces, energies, potentials
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", SMALL)
def test_force_energy_potential_match_oracle(precision, name):
    w = WORKLOADS[name]
    pos, q = positions_charges(w.N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, precision)
    s = osys(m, w)
    k = m.sample_k(0, return_k=True).cpu().numpy()
    F, phi, e = m.force(dev(pos), dev(q), energy=True, potential=True)
    ref = O.rbe(s, pos, q, k, mode=1, want_dq=True)
    print(f"{name} {precision}: force rel-L2 = {rel_l2(F.cpu().numpy(), ref['force']):.3e}, "
          f"phi rel-L2 = {rel_l2(phi.cpu().numpy(), ref['dUdq']):.3e}")
    assert rel_l2(F.cpu().numpy(), ref["force"]) < TOL[precision]
    assert rel_l2(phi.cpu().numpy(), ref["dUdq"]) < TOL[precision]
    e = e.cpu().numpy()
    for i in range(3):
        assert e[i] == pytest.approx(ref["energy"][i], rel=TOL[precision], abs=1e-9 * abs(ref["energy"]).max())
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_force_with_explicit_batch_and_explicit_images(precision):
    """An explicit batch (rbe2d_set_k) and the oracle's explicit-image definition
    (Eq. 3.17, no re-calibration), with a ragged N and an asymmetric dielectric."""
    from paper_2405_06333_gb300.rbe2d import RBE2D
    N, P = 777, 64
    pos, q = positions_charges(N, 12.0, 9.0, 3.0, seed=21)
    q[-1] = -np.sum(q[:-1])
    m = RBE2D(12.0, 9.0, 3.0, n_max=N, P=P, gamma_top=-0.7, gamma_bot=0.45, M=6, Lz=-1, alpha=0.9,
              precision=precision)
    s = osys(m, type("W", (), dict(Lx=12.0, Ly=9.0, H=3.0, gamma_top=-0.7, gamma_bot=0.45))())
    k = random_kbatch(P, nmax=(6, 6, 40), seed=3)
    m.set_k(k)
    F, phi, e = m.force(dev(pos), dev(q), energy=True, potential=True)
    ref = O.rbe(s, pos, q, k, mode=0, want_dq=True)
    assert rel_l2(F.cpu().numpy(), ref["force"]) < TOL[precision]
    assert rel_l2(phi.cpu().numpy(), ref["dUdq"]) < TOL[precision]
    assert e.cpu().numpy()[0] == pytest.approx(ref["energy"][0], rel=TOL[precision])
    m.sync_status()
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["slab_n1e6", "thin_n1e6"])
def test_full_size_sampled_targets(precision, name):
    """N = 1e6, P = 500 in the launch shape the benchmark times: every force is computed
    on the GPU; the oracle computes the full structure factors and the forces of 1500
    sampled particles (plus the first and last few, covering the ragged chunk ends)."""
    w = WORKLOADS[name]
    pos, q = positions_charges(w.N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, precision)
    s = osys(m, w)
    k = m.sample_k(0, return_k=True).cpu().numpy()
    F, e = m.force(dev(pos), dev(q), energy=True)
    rng = np.random.default_rng(17)
    tg = np.unique(np.concatenate([rng.choice(w.N, 1500, replace=False), np.arange(8), w.N - 1 - np.arange(8)]))
    ref = O.rbe(s, pos, q, k, mode=1, targets=tg)
    err = rel_l2(F.cpu().numpy()[tg], ref["force"])
    print(f"{name} {precision}: force rel-L2 = {err:.3e}, U_k rel = {abs(e[0].item() / ref['energy'][0] - 1):.3e}")
    assert err < TOL[precision]
    assert e.cpu().numpy()[0] == pytest.approx(ref["energy"][0], rel=TOL[precision])
    assert e.cpu().numpy()[2] == pytest.approx(ref["energy"][2], rel=TOL[precision], abs=1e-9)
    m.close()


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_matches_oracle_gradient(precision):
    w = WORKLOADS["adjoint_n1e5"]
    N = 20000
    pos, q = positions_charges(N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, precision, n_max=N)
    s = osys(m, w)
    k = m.sample_k(0, return_k=True).cpu().numpy()
    g = 0.75
    dpos, dq, dg = m.energy_backward(dev(pos), dev(q), g)
    tg = np.arange(0, N, 7)
    ref = O.rbe(s, pos, q, k, mode=1, targets=tg, want_dq=True, want_dgamma=True)
    assert rel_l2(dpos.cpu().numpy()[tg], -g * ref["force"]) < TOL[precision]
    assert rel_l2(dq.cpu().numpy()[tg], g * ref["dUdq"]) < TOL[precision]
    assert rel_l2(dg.cpu().numpy(), g * ref["dUdgamma"]) < TOL[precision]
    m.close()


def test_autograd_function_fd_and_oracle():
    """torch.autograd through RBE2DEnergy (FP64 mode): gradients w.r.t. positions,
    charges and both gammas equal central finite differences (h = 1e-4) of the GPU
    energy on a fixed batch, and the oracle gradient."""
    from paper_2405_06333_gb300.rbe2d import RBE2DEnergy
    w = WORKLOADS["adjoint_n1e5"]
    N = 4000
    pos, q = positions_charges(N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, "fp64", n_max=N)
    m.sample_k(0)
    P_ = dev(pos).requires_grad_(True)
    Q_ = dev(q).requires_grad_(True)
    G_ = torch.tensor([w.gamma_top, w.gamma_bot], dtype=torch.float64, device="cuda", requires_grad=True)
    U = RBE2DEnergy.apply(m, P_, Q_, G_)
    U.backward()
    h = 1e-4
    def energy(p, qq):
        _, e = m.force(dev(p), dev(qq), energy=True)
        return float(e[:3].sum())
    for i, d in [(0, 0), (5, 2), (123, 1)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[i, d] += h; p2[i, d] -= h
        fd = (energy(p1, q) - energy(p2, q)) / (2 * h)
        assert float(P_.grad[i, d]) == pytest.approx(fd, rel=1e-5, abs=1e-7)
    for i in (3, 77):
        q1, q2 = q.copy(), q.copy()
        q1[i] += h; q2[i] -= h
        fd = (energy(pos, q1) - energy(pos, q2)) / (2 * h)
        assert float(Q_.grad[i]) == pytest.approx(fd, rel=1e-5, abs=1e-7)
    from paper_2405_06333_gb300.rbe2d import RBE2D
    for j, name in enumerate(("gamma_top", "gamma_bot")):
        es = []
        for sg in (+1, -1):
            gg = dict(gamma_top=w.gamma_top, gamma_bot=w.gamma_bot)
            gg[name] += sg * h
            mm = RBE2D(w.Lx, w.Ly, w.H, n_max=N, P=w.P, M=m.derived["M"], Lz=m.derived["Lz"],
                       alpha=m.derived["alpha"], seed=w.seed, precision="fp64", **gg)
            mm.sample_k(0)
            _, e = mm.force(dev(pos), dev(q), energy=True)
            es.append(float(e[:3].sum()))
            mm.close()
        fd = (es[0] - es[1]) / (2 * h)
        assert float(G_.grad[j]) == pytest.approx(fd, rel=1e-5, abs=1e-7)
    m.close()


# ------------------------------------------------------------------ edge cases and errors
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_cases(precision):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    # N = 0: nothing to do, no error
    m = RBE2D(10.0, 10.0, 2.0, n_max=8, P=1, gamma_top=0.0, gamma_bot=0.6, M=1, Lz=-1, alpha=1.0,
              precision=precision)
    m.sample_k(0)
    F = m.force(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert F.shape == (0, 3)
    # a neutral pair at the interfaces and on the cell edge, P = 1, a single interface
    pos = np.array([[10.0, 0.0, 0.0], [3.0, 9.999999, 2.0]])
    q = np.array([1.0, -1.0])
    s = osys(m, type("W", (), dict(Lx=10.0, Ly=10.0, H=2.0, gamma_top=0.0, gamma_bot=0.6))())
    for step in range(4):
        k = m.sample_k(step, return_k=True).cpu().numpy()
        F, e = m.force(dev(pos), dev(q), energy=True)
        ref = O.rbe(s, pos, q, k, mode=0)
        assert rel_l2(F.cpu().numpy(), ref["force"]) < TOL[precision]
    # x, y outside the cell are wrapped: same forces as the wrapped positions
    wrapped = pos.copy(); wrapped[:, 0] = np.mod(pos[:, 0], 10.0); wrapped[:, 1] = np.mod(pos[:, 1], 10.0)
    shifted = wrapped.copy(); shifted[:, 0] += np.array([-20.0, 30.0]); shifted[:, 1] -= 10.0
    Fa = m.force(dev(wrapped), dev(q)).cpu().numpy()
    Fb = m.force(dev(shifted), dev(q)).cpu().numpy()
    assert rel_l2(Fb, Fa) < TOL[precision]
    m.close()
    # |gamma| = 1 with a capped image series
    m = RBE2D(8.0, 8.0, 4.0, n_max=64, P=50, gamma_top=1.0, gamma_bot=-1.0, M=-1, Lz=-1, alpha=1.0,
              precision=precision)
    assert 1 <= m.derived["M"] <= 64
    pos, q = positions_charges(64, 8.0, 8.0, 4.0, seed=9)
    k = m.sample_k(1, return_k=True).cpu().numpy()
    F = m.force(dev(pos), dev(q)).cpu().numpy()
    s = osys(m, type("W", (), dict(Lx=8.0, Ly=8.0, H=4.0, gamma_top=1.0, gamma_bot=-1.0))())
    assert rel_l2(F, O.rbe(s, pos, q, k, mode=1)["force"]) < TOL[precision]
    m.close()


def test_error_codes():
    from paper_2405_06333_gb300.rbe2d import RBE2D
    m = RBE2D(10.0, 10.0, 2.0, n_max=100, P=16, gamma_top=0.3, gamma_bot=0.2, M=3, Lz=-1, alpha=1.0,
              precision="fp32")
    pos, q = positions_charges(100, 10.0, 10.0, 2.0, seed=1)
    # no batch yet
    F = torch.empty((100, 3), device="cuda")
    code = B.status_code(B.rbe2d_force, m.ctx, 100, dev(pos), dev(q), B.RBE2D_KSPACE, F)
    assert code == B.RBE2D_EINVAL
    m.sample_k(0)
    # N > n_max
    code = B.status_code(B.rbe2d_force, m.ctx, 101, dev(np.zeros((101, 3))), dev(np.zeros(101)), B.RBE2D_KSPACE, F)
    assert code == B.RBE2D_EINVAL
    # non-neutral, checked on request
    q2 = q.copy(); q2[0] += 0.5
    code = B.status_code(B.rbe2d_force, m.ctx, 100, dev(pos), dev(q2), B.RBE2D_KSPACE | B.RBE2D_VALIDATE, F)
    assert code == B.RBE2D_ENONNEUTRAL
    # z outside the slab, checked on request
    p2 = pos.copy(); p2[3, 2] = 2.5
    code = B.status_code(B.rbe2d_force, m.ctx, 100, dev(p2), dev(q), B.RBE2D_KSPACE | B.RBE2D_VALIDATE, F)
    assert code == B.RBE2D_ERANGE
    # valid input passes validation; messages are set on failure
    assert B.status_code(B.rbe2d_force, m.ctx, 100, dev(pos), dev(q), B.RBE2D_KSPACE | B.RBE2D_VALIDATE, F) == 0
    # explicit batch with a k = 0 row is reported by rbe2d_sync_status
    kz = torch.zeros((16, 3), dtype=torch.int32, device="cuda"); kz[:, 2] = 1; kz[5] = 0
    B.rbe2d_set_k(m.ctx, kz)
    assert B.status_code(B.rbe2d_sync_status, m.ctx) == B.RBE2D_ESAMPLER
    assert "k = 0" in B.rbe2d_last_error(m.ctx)
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_validate_accepts_charges_on_both_interfaces(precision):
    """z = 0 and z = H are inside the slab even when H has no exact float32 value (the
    range check compares float64 extrema); a charge just above H is out."""
    from paper_2405_06333_gb300.rbe2d import RBE2D
    H = 0.1
    N = 1000
    m = RBE2D(5.0, 5.0, H, n_max=N, P=16, gamma_top=0.3, gamma_bot=0.2, M=3, Lz=-1, alpha=2.0, precision=precision)
    pos, q = positions_charges(N, 5.0, 5.0, H, seed=2)
    pos[0, 2] = H
    pos[1, 2] = 0.0
    pos[2, 2] = H
    m.sample_k(0)
    F = torch.empty((N, 3), dtype=m.out_dtype, device="cuda")
    fl = B.RBE2D_KSPACE | B.RBE2D_VALIDATE
    assert B.status_code(B.rbe2d_force, m.ctx, N, dev(pos), dev(q), fl, F) == B.RBE2D_OK
    pos[2, 2] = np.nextafter(H, 1.0)
    assert B.status_code(B.rbe2d_force, m.ctx, N, dev(pos), dev(q), fl, F) == B.RBE2D_ERANGE
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_host_buffers_f32_inputs_determinism_and_reuse(precision):
    w = WORKLOADS["dielectric_n1e4"]
    pos, q = positions_charges(w.N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, precision)
    m.sample_k(7)
    F1, e1 = m.force(dev(pos), dev(q), energy=True)
    F2, e2 = m.force(dev(pos), dev(q), energy=True)
    assert torch.equal(F1, F2) and torch.equal(e1, e2)  # bitwise reproducible
    F3 = m.force(dev(pos), dev(q), reuse_sf=True)
    assert torch.equal(F1, F3)
    # host buffers through the same C entry point
    odt = np.float64 if precision == "fp64" else np.float32
    Fh = np.zeros((w.N, 3), dtype=odt)
    eh = np.zeros(4)
    B.rbe2d_force(m.ctx, w.N, np.ascontiguousarray(pos), np.ascontiguousarray(q),
                  B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY | B.RBE2D_HOST_BUFFERS, Fh, None, eh)
    assert np.array_equal(Fh, F1.cpu().numpy())
    assert np.array_equal(eh, e1.cpu().numpy())
    # float32 inputs
    F4 = m.force(dev(pos, torch.float32), dev(q, torch.float32))
    assert rel_l2(F4.cpu().numpy(), F1.cpu().numpy()) < (1e-5 if precision == "fp64" else 1e-4)
    m.close()


def test_sampling_is_unbiased_on_gpu():
    """The GPU estimator averaged over steps approaches the oracle's full k-sum force
    (Theorem 2.3); each component within 5 standard errors."""
    from paper_2405_06333_gb300.rbe2d import RBE2D
    Lx, Ly, H = 8.0, 8.0, 2.0
    pos, q = positions_charges(10, Lx, Ly, H, seed=12)
    m = RBE2D(Lx, Ly, H, n_max=10, P=20, gamma_top=0.7, gamma_bot=-0.5, M=4, Lz=24.0, alpha=0.6, precision="fp64")
    s = osys(m, type("W", (), dict(Lx=Lx, Ly=Ly, H=H, gamma_top=0.7, gamma_bot=-0.5))())
    nm = [O.nmax(s.alpha, L) for L in (s.Lx, s.Ly, s.Lz)]
    kf, wf = O.full_klist(s, nm)
    Ff = O.kspace(s, pos, q, kf, wf, mode=1)["force"]
    Fs = []
    for step in range(600):
        m.sample_k(step)
        Fs.append(m.force(dev(pos), dev(q)).cpu().numpy())
    Fs = np.stack(Fs)
    se = Fs.std(0, ddof=1) / np.sqrt(len(Fs))
    assert np.all(np.abs(Fs.mean(0) - Ff) < 5 * se + 1e-12)
    m.close()


@pytest.mark.parametrize("name,N", [("dielectric_n1e4", 3001), ("plain_n1e3", 999)])
def test_every_force_shape_at_a_ragged_small_size(name, N):
    """Each force shape, including those that split a particle's k-sum over 2 or 4 threads,
    on a small odd N (the last round partly empty, idle lanes in the shuffles), with and
    without the dielectric term: forces and potential against the oracle."""
    w = WORKLOADS[name]
    pos, q = positions_charges(N, w.Lx, w.Ly, w.H, seed=w.pos_seed)  # odd N: one uncharged particle
    m = make(w, "fp32", n_max=N)
    s = osys(m, w)
    k = m.sample_k(1, return_k=True).cpu().numpy()
    ref = O.rbe(s, pos, q, k, mode=1)["force"]
    P_, Q_ = dev(pos), dev(q)
    for fshape in range(7):
        B.rbe2d_set_tuning(m.ctx, 2, 1, 0, fshape)
        F = m.force(P_, Q_)
        err = rel_l2(F.cpu().numpy(), ref)
        assert err < TOL["fp32"], (name, fshape, err)
    m.close()


def test_tuner_variants_keep_parity():
    """Every variant the autotuner can pick (FMA-pipe share of the sin/cos x the
    structure factor's shape x the force kernel's round shape) meets the FP32 bar at the
    full size, and the autotuner returns one of them, which meets it too."""
    w = WORKLOADS["slab_n1e6"]
    pos, q = positions_charges(w.N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, "fp32")
    s = osys(m, w)
    k = m.sample_k(0, return_k=True).cpu().numpy()
    tg = np.random.default_rng(5).choice(w.N, 800, replace=False)
    ref = O.rbe(s, pos, q, k, mode=1, targets=tg)["force"]
    P_, Q_ = dev(pos), dev(q)
    for poly in (0, 1, 2, 3):
        for fshape in range(7):
            sfshape = fshape % 3
            B.rbe2d_set_tuning(m.ctx, poly, poly, sfshape, fshape)
            F = m.force(P_, Q_)
            err = rel_l2(F.cpu().numpy()[tg], ref)
            print(f"poly {poly} sf shape {sfshape} force shape {fshape}: force rel-L2 = {err:.3e}")
            assert err < TOL["fp32"], (poly, sfshape, fshape)
    with pytest.raises(B.RBE2DError):
        B.rbe2d_set_tuning(m.ctx, 0, 0, 3, 0)
    with pytest.raises(B.RBE2DError):
        B.rbe2d_set_tuning(m.ctx, 4, 0, 0, 0)
    with pytest.raises(B.RBE2DError):
        B.rbe2d_set_tuning(m.ctx, 0, 0, 0, 7)
    ch = B.rbe2d_autotune(m.ctx, w.N, P_, Q_, B.RBE2D_IBC, torch.empty((w.N, 3), device="cuda"))
    assert ch["sf_poly"] in (0, 1, 2, 3) and ch["force_poly"] in (0, 1, 2, 3)
    assert ch["sf_shape"] in (0, 1, 2) and ch["force_shape"] in range(7)
    F = m.force(P_, Q_)
    assert rel_l2(F.cpu().numpy()[tg], ref) < TOL["fp32"]
    m.close()
