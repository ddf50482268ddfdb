"""GPU parity of the energy adjoint and of the potential at the workloads' full sizes.

The adjoint of the random-batch k-space energy U = U_k + U_self + U_IBC (Theorem 3.3,
Eq. 3.16 with the estimator of Sec. 2.3 and the re-calibrated images of Sec. 3.4) is
compared element by element with the FP64 oracle on the same k batch:
  dpos = g dU/dr_i = -g F_i,  dq = g dU/dq_i,  dgamma = g (dU/dgamma_top, dU/dgamma_bot).
The sizes are the ones the benchmark and the adjoint workload run at, so the force
kernel takes many rounds per CTA (N = 1e6: 1954 rounds of 512 particles over 760 CTAs),
which the smaller parity tests never reach.

Bars (written here, from the build's target): relative L2 error over all compared
components <= 1e-5 in RBE2D_FP64 mode and <= 1e-4 in RBE2D_FP32_MIXED mode.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300.synthetic import WORKLOADS, positions_charges

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-5, "fp32": 1e-4}
G = 0.75  # upstream gradient of the energy


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


def make(w, precision):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    return RBE2D(w.Lx, w.Ly, w.H, n_max=w.N, P=w.P, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M,
                 Lz=w.Lz, alpha=w.alpha, r_c=w.r_c, seed=w.seed, precision=precision)


def osys(w, model):
    d = model.derived
    return O.System(Lx=w.Lx, Ly=w.Ly, H=w.H, Lz=d["Lz"], gamma_top=w.gamma_top, gamma_bot=w.gamma_bot,
                    alpha=d["alpha"], M=d["M"])


def targets_of(name):
    w = WORKLOADS[name]
    if w.N <= 100000:
        return np.arange(w.N)  # every particle
    rng = np.random.default_rng(29)
    # 1500 sampled particles plus both ends (the first and the last, partial, round)
    return np.unique(np.concatenate([rng.choice(w.N, 1500, replace=False), np.arange(8),
                                     w.N - 1 - np.arange(8)]))


@functools.lru_cache(maxsize=None)
def reference(name):
    """Inputs, the step-0 batch and the oracle's energy, force, dU/dq and dU/dgamma on the
    targets (computed once per workload and shared by the precisions)."""
    w = WORKLOADS[name]
    pos, q = positions_charges(w.N, w.Lx, w.Ly, w.H, seed=w.pos_seed)
    m = make(w, "fp64")
    s = osys(w, m)
    k = m.sample_k(0, return_k=True).cpu().numpy()
    m.close()
    assert np.array_equal(k, O.sample_k(s, w.seed, 0, w.P))
    tg = targets_of(name)
    ref = O.rbe(s, pos, q, k, mode=1, targets=tg, want_dq=True, want_dgamma=True)
    return pos, q, k, tg, ref


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["slab_n1e6", "adjoint_n1e5"])
def test_energy_backward_full_size(precision, name):
    w = WORKLOADS[name]
    pos, q, k, tg, ref = reference(name)
    m = make(w, precision)
    m.sample_k(0)
    dpos, dq, dg = m.energy_backward(dev(pos), dev(q), G)
    torch.cuda.synchronize()
    m.sync_status()
    e_dpos = rel_l2(dpos.cpu().numpy()[tg], -G * ref["force"])
    e_dq = rel_l2(dq.cpu().numpy()[tg], G * ref["dUdq"])
    e_dg = rel_l2(dg.cpu().numpy(), G * ref["dUdgamma"])
    print(f"{name} {precision}: dpos {e_dpos:.3e}  dq {e_dq:.3e}  dgamma {e_dg:.3e} "
          f"({len(tg)} targets)")
    assert e_dpos < TOL[precision]
    assert e_dq < TOL[precision]
    assert e_dg < TOL[precision]
    # each gamma derivative on its own, not only the pair's norm
    for j in range(2):
        assert float(dg[j]) == pytest.approx(G * ref["dUdgamma"][j], rel=TOL[precision])
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_potential_full_size(precision):
    """rbe2d_force with RBE2D_POTENTIAL at N = 1e6, P = 500: the force and dU/dq of the
    same launch (the potential variant of the force kernel over many rounds per CTA)."""
    name = "slab_n1e6"
    w = WORKLOADS[name]
    pos, q, k, tg, ref = reference(name)
    m = make(w, precision)
    m.sample_k(0)
    F, phi, e = m.force(dev(pos), dev(q), energy=True, potential=True)
    torch.cuda.synchronize()
    e_f = rel_l2(F.cpu().numpy()[tg], ref["force"])
    e_p = rel_l2(phi.cpu().numpy()[tg], ref["dUdq"])
    print(f"{name} {precision}: force {e_f:.3e}  phi {e_p:.3e}")
    assert e_f < TOL[precision]
    assert e_p < TOL[precision]
    e = e.cpu().numpy()
    for i in range(3):
        assert e[i] == pytest.approx(ref["energy"][i], rel=TOL[precision], abs=1e-9 * abs(ref["energy"]).max())
    m.close()


@pytest.mark.parametrize("name", ["slab_n1e6", "adjoint_n1e5"])
def test_potential_tuner_variants_keep_parity(name):
    """Every variant of the force kernel's potential variant (FMA-pipe share x round
    shape: 256 x 2 with the k-sum in 1, 2 or 4 threads, 256 x 1) gives the force and dU/dq
    within the FP32 bar at full size, through rbe2d_force and rbe2d_energy_backward, and
    the potential autotuner returns one of them."""
    from paper_2405_06333_gb300 import binding as B
    w = WORKLOADS[name]
    pos, q, k, tg, ref = reference(name)
    m = make(w, "fp32")
    m.sample_k(0)
    P_, Q_ = dev(pos), dev(q)
    for poly in range(4):
        for shape in range(4):
            B.rbe2d_set_tuning_potential(m.ctx, poly, shape)
            F, phi = m.force(P_, Q_, potential=True)
            e_f = rel_l2(F.cpu().numpy()[tg], ref["force"])
            e_p = rel_l2(phi.cpu().numpy()[tg], ref["dUdq"])
            dpos, dq, _ = m.energy_backward(P_, Q_, G, reuse_sf=True)
            e_b = rel_l2(dq.cpu().numpy()[tg], G * ref["dUdq"])
            print(f"{name} poly {poly} shape {shape}: force {e_f:.3e} phi {e_p:.3e} backward dq {e_b:.3e}")
            assert max(e_f, e_p, e_b) < TOL["fp32"], (poly, shape, e_f, e_p, e_b)
            assert rel_l2(dpos.cpu().numpy()[tg], -G * ref["force"]) < TOL["fp32"]
    with pytest.raises(B.RBE2DError):
        B.rbe2d_set_tuning_potential(m.ctx, 0, 4)
    with pytest.raises(B.RBE2DError):
        B.rbe2d_set_tuning_potential(m.ctx, 4, 0)
    ch = B.rbe2d_autotune_potential(m.ctx, w.N, P_, Q_, B.RBE2D_IBC, torch.empty((w.N, 3), device="cuda"),
                                    torch.empty(w.N, device="cuda"))
    print(name, ch)
    assert ch["potential_poly"] in range(4) and ch["potential_shape"] in range(4)
    _, phi = m.force(P_, Q_, potential=True)
    assert rel_l2(phi.cpu().numpy()[tg], ref["dUdq"]) < TOL["fp32"]
    m.sync_status()
    m.close()


def test_autograd_fp32_adjoint_workload():
    """torch.autograd through RBE2DEnergy in FP32-mixed mode at the adjoint workload's
    full size (N = 1e5, P = 300): the gradients with respect to every position, every
    charge and both contrasts against the oracle gradient."""
    from paper_2405_06333_gb300.rbe2d import RBE2DEnergy
    name = "adjoint_n1e5"
    w = WORKLOADS[name]
    pos, q, k, tg, ref = reference(name)
    m = make(w, "fp32")
    m.sample_k(0)
    P_ = dev(pos).requires_grad_(True)
    Q_ = dev(q).requires_grad_(True)
    G_ = torch.tensor([w.gamma_top, w.gamma_bot], dtype=torch.float64, device="cuda", requires_grad=True)
    U = RBE2DEnergy.apply(m, P_, Q_, G_)
    (G * U).backward()
    U_ref = float(np.sum(ref["energy"]))
    assert float(U) == pytest.approx(U_ref, rel=TOL["fp32"], abs=1e-7 * abs(ref["energy"]).max())
    e_dpos = rel_l2(P_.grad.cpu().numpy()[tg], -G * ref["force"])
    e_dq = rel_l2(Q_.grad.cpu().numpy()[tg], G * ref["dUdq"])
    e_dg = rel_l2(G_.grad.cpu().numpy(), G * ref["dUdgamma"])
    print(f"autograd fp32: dpos {e_dpos:.3e}  dq {e_dq:.3e}  dgamma {e_dg:.3e}")
    assert e_dpos < TOL["fp32"] and e_dq < TOL["fp32"] and e_dg < TOL["fp32"]
    m.close()
