"""Per-sample invariants of the GPU k-space force on one explicit batch (rbe2d_set_k), in
both precisions, with a ragged N and a batch that is not a multiple of any tile:

- sum_i F_x = sum_i F_y = 0: the batch estimator of Eq. 3.26 is a sum over k of terms
  c k Im(conj(rho) A + conj(sigma) B), and with A = (2 + 2E) rho + conj(O) sigma,
  B = O rho each of them is real (E real; the two cross terms are complex conjugates);
- with gamma = 0 also sum_i F_z = 0 (no images; the IBC force of Eq. 3.18 is
  proportional to q_i and the system is neutral);
- a translation in x and y leaves forces and energies unchanged (periodic cell), and a
  particle at x = Lx or y = Ly acts as one at 0;
- the mirror z -> H - z with gamma_top <-> gamma_bot and n_z -> -n_z maps the force to
  (F_x, F_y, -F_z) and leaves the energies unchanged.

These hold in exact arithmetic for every batch; the tolerances are the rounding of each
mode (float64 throughout; float32 phases and products)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2405_06333_gb300.synthetic import positions_charges, random_kbatch

pytestmark = pytest.mark.gpu

# cancellation in a sum of N forces: relative to sum |F|; agreement of two evaluations: rel-L2
SUM_TOL = {"fp64": 1e-11, "fp32": 2e-5}
EQ_TOL = {"fp64": 1e-11, "fp32": 2e-5}


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


def run(precision, pos, q, k, gt, gb, M, Lx=12.0, Ly=9.0, H=3.0):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    m = RBE2D(Lx, Ly, H, n_max=len(q), P=k.shape[0], gamma_top=gt, gamma_bot=gb, M=M, Lz=40.0, alpha=0.9,
              precision=precision)
    m.set_k(k)
    F, e = m.force(torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"), energy=True)
    out = F.double().cpu().numpy(), e.cpu().numpy()
    m.sync_status()
    m.close()
    return out


N, P = 2001, 97


def inputs(seed=31):
    pos, q = positions_charges(N, 12.0, 9.0, 3.0, seed=seed)
    return pos, q, random_kbatch(P, nmax=(7, 6, 45), seed=seed + 1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_net_force_vanishes_in_x_and_y(precision):
    pos, q, k = inputs()
    F, _ = run(precision, pos, q, k, -0.6, 0.85, 6)
    for d in (0, 1):
        assert abs(F[:, d].sum()) < SUM_TOL[precision] * np.abs(F[:, d]).sum(), d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_net_force_vanishes_without_images(precision):
    pos, q, k = inputs(seed=32)
    F, _ = run(precision, pos, q, k, 0.0, 0.0, 0)
    for d in range(3):
        assert abs(F[:, d].sum()) < SUM_TOL[precision] * np.abs(F[:, d]).sum(), d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_xy_translation_and_cell_edges(precision):
    pos, q, k = inputs(seed=33)
    F, e = run(precision, pos, q, k, -0.6, 0.85, 6)
    sh = pos.copy()
    sh[:, 0] += 3.7
    sh[:, 1] -= 1.3  # partly negative: wrapped by the fixed-point phases
    Fs, es = run(precision, sh, q, k, -0.6, 0.85, 6)
    assert rel_l2(Fs, F) < EQ_TOL[precision]
    assert es[:3] == pytest.approx(e[:3], rel=EQ_TOL[precision], abs=1e-12)
    edge = pos.copy()
    edge[:5, 0] = 0.0
    edge[5:10, 1] = 0.0
    Fa, _ = run(precision, edge, q, k, -0.6, 0.85, 6)
    edge[:5, 0] = 12.0
    edge[5:10, 1] = 9.0
    Fb, _ = run(precision, edge, q, k, -0.6, 0.85, 6)
    assert rel_l2(Fb, Fa) < EQ_TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_z_mirror_with_swapped_contrasts(precision):
    pos, q, k = inputs(seed=34)
    F, e = run(precision, pos, q, k, -0.6, 0.85, 6)
    mp = pos.copy()
    mp[:, 2] = 3.0 - pos[:, 2]
    km = k.copy()
    km[:, 2] *= -1
    Fm, em = run(precision, mp, q, km, 0.85, -0.6, 6)
    assert rel_l2(Fm * [1.0, 1.0, -1.0], F) < EQ_TOL[precision]
    assert em[:3] == pytest.approx(e[:3], rel=EQ_TOL[precision], abs=1e-12)
