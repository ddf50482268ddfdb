"""GPU parity of the cell-list real-space part with image charges (Eq. 3.12, reading
A15) against the oracle's brute-force sum over all pairs, replicas and images.

Bars as for the k-space path: force rel-L2 <= 1e-5 (FP64 mode) / 1e-4 (FP32 mode);
energy relative error within the same bounds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import positions_charges

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


def model(Lx, Ly, H, N, precision, gt, gb, M, alpha, r_c, P=16):
    p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=-1, gamma_top=gt, gamma_bot=gb, M=M, alpha=alpha, r_c=r_c, P=P,
                       seed=0, eps=1e-4, precision=B.RBE2D_FP64 if precision == "fp64" else B.RBE2D_FP32_MIXED,
                       coulomb_k=1.0, real_space=1)
    ctx = B.rbe2d_init(p, N, torch.cuda.current_stream())
    B.rbe2d_sample_k(ctx, 0, None)
    return ctx


def real_only(ctx, N, pos, q, precision, energy=False, potential=False):
    dt = torch.float64 if precision == "fp64" else torch.float32
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    phi = torch.empty(N, dtype=dt, device="cuda") if potential else None
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    fl = B.RBE2D_REAL | (B.RBE2D_ENERGY if energy else 0) | (B.RBE2D_POTENTIAL if potential else 0)
    B.rbe2d_force(ctx, N, dev(pos), dev(q), fl, F, phi, e)
    torch.cuda.synchronize()
    return F.cpu().numpy(), e.cpu().numpy(), (phi.cpu().numpy() if potential else None)


CASES = [
    # (Lx, Ly, H, N, gt, gb, M, alpha, r_c): thick slab with thin image shells; thin slab
    # with H < r_c (several image levels within r_c); small box with r_c > Lx/2
    (40.0, 40.0, 5.0, 10000, -0.95, -0.95, 20, 0.3, 8.0),
    (63.0, 63.0, 20.0, 100000, 0.9, -0.9, 14, 1.0772173450159417, 2.785),
    (7.0, 9.0, 3.0, 300, 0.6, -0.4, 6, 0.7, 6.0),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_real_space_force_matches_oracle(precision, case):
    Lx, Ly, H, N, gt, gb, M, a, rc = CASES[case]
    pos, q = positions_charges(N, Lx, Ly, H, seed=40 + case)
    ctx = model(Lx, Ly, H, N, precision, gt, gb, M, a, rc)
    F, _, _ = real_only(ctx, N, pos, q, precision)
    s = O.System(Lx=Lx, Ly=Ly, H=H, Lz=1e9, gamma_top=gt, gamma_bot=gb, alpha=a, M=M)
    rng = np.random.default_rng(3)
    tg = np.unique(np.concatenate([rng.choice(N, min(N, 300), replace=False), [0, N - 1]]))
    Fo, _ = O.real_space(s, rc, pos, q, targets=tg)
    err = rel_l2(F[tg], Fo)
    print(f"case {case} {precision}: real-space force rel-L2 = {err:.3e}")
    assert err < TOL[precision]
    B.rbe2d_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_real_space_energy_and_potential(precision):
    Lx, Ly, H, N = 20.0, 20.0, 4.0, 2000
    gt, gb, M, a, rc = -0.8, 0.5, 8, 0.8, 5.0
    pos, q = positions_charges(N, Lx, Ly, H, seed=7)
    ctx = model(Lx, Ly, H, N, precision, gt, gb, M, a, rc)
    F, e, _ = real_only(ctx, N, pos, q, precision, energy=True)
    s = O.System(Lx=Lx, Ly=Ly, H=H, Lz=1e9, gamma_top=gt, gamma_bot=gb, alpha=a, M=M)
    Fo, Uo = O.real_space(s, rc, pos, q)
    assert rel_l2(F, Fo) < TOL[precision]
    assert e[3] == pytest.approx(Uo, rel=TOL[precision])
    # dU_real/dq_i by central differences of the oracle energy
    _, _, phi = real_only(ctx, N, pos, q, precision, potential=True)
    h = 1e-5
    for i in (0, 999, 1500):
        q1, q2 = q.copy(), q.copy()
        q1[i] += h; q2[i] -= h
        fd = (O.real_space(s, rc, pos, q1)[1] - O.real_space(s, rc, pos, q2)[1]) / (2 * h)
        assert phi[i] == pytest.approx(fd, rel=10 * TOL[precision], abs=1e-6)
    B.rbe2d_destroy(ctx)


def test_total_force_is_kspace_plus_real_and_reproducible():
    """RBE2D_KSPACE | RBE2D_IBC | RBE2D_REAL equals the k-space force plus the real-space
    force, and two calls agree bit for bit."""
    Lx, Ly, H, N = 30.0, 30.0, 6.0, 5000
    pos, q = positions_charges(N, Lx, Ly, H, seed=8)
    ctx = model(Lx, Ly, H, N, "fp32", 0.7, -0.3, 6, 0.9, 3.5, P=64)
    F = torch.empty((N, 3), device="cuda")
    Fk = torch.empty((N, 3), device="cuda")
    Fr = torch.empty((N, 3), device="cuda")
    B.rbe2d_force(ctx, N, dev(pos), dev(q), B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL, F)
    F2 = torch.empty_like(F)
    B.rbe2d_force(ctx, N, dev(pos), dev(q), B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL, F2)
    B.rbe2d_force(ctx, N, dev(pos), dev(q), B.RBE2D_KSPACE | B.RBE2D_IBC, Fk)
    B.rbe2d_force(ctx, N, dev(pos), dev(q), B.RBE2D_REAL, Fr)
    torch.cuda.synchronize()
    assert torch.equal(F, F2)
    assert rel_l2(F.cpu().numpy(), (Fk + Fr).cpu().numpy()) < 1e-6
    B.rbe2d_destroy(ctx)


def test_real_space_needs_the_cell_list():
    p = B.rbe2d_params(Lx=10, Ly=10, H=2, Lz=-1, gamma_top=0, gamma_bot=0, M=0, alpha=1.0, r_c=3.0, P=8, seed=0,
                       eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=0)
    ctx = B.rbe2d_init(p, 10, torch.cuda.current_stream())
    B.rbe2d_sample_k(ctx, 0, None)
    F = torch.empty((10, 3), device="cuda")
    code = B.status_code(B.rbe2d_force, ctx, 10, dev(np.zeros((10, 3))), dev(np.zeros(10)), B.RBE2D_REAL, F)
    assert code == B.RBE2D_EINVAL
    B.rbe2d_destroy(ctx)


def test_real_space_energy_slot_is_cleared_without_real():
    """energy_out[3] holds the real-space energy only for calls with RBE2D_REAL; a later
    call without it (with or without reusing the structure factors) reports 0 there."""
    Lx, Ly, H, N = 30.0, 30.0, 6.0, 3000
    pos, q = positions_charges(N, Lx, Ly, H, seed=9)
    ctx = model(Lx, Ly, H, N, "fp32", 0.7, -0.3, 6, 0.9, 3.5, P=32)
    F = torch.empty((N, 3), device="cuda")
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    P_, Q_ = dev(pos), dev(q)
    base = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY
    B.rbe2d_force(ctx, N, P_, Q_, base | B.RBE2D_REAL, F, None, e)
    torch.cuda.synchronize()
    assert e[3].item() != 0.0
    B.rbe2d_force(ctx, N, P_, Q_, base | B.RBE2D_REUSE_SF, F, None, e)
    torch.cuda.synchronize()
    assert e[3].item() == 0.0
    B.rbe2d_force(ctx, N, P_, Q_, base | B.RBE2D_REAL | B.RBE2D_REUSE_SF, F, None, e)
    B.rbe2d_force(ctx, N, P_, Q_, base, F, None, e)
    torch.cuda.synchronize()
    assert e[3].item() == 0.0
    B.rbe2d_destroy(ctx)
