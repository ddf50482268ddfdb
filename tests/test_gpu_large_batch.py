"""Large k batches against the oracle's explicit-image definition (Eq. 3.17, no
re-calibration), both precisions: P = 600 splits the structure factor over two k-chunks
of 512, P = 2501 over five and the float32 force over three shared-memory tiles of 1024
wave vectors, the last one odd (its final record has one wave vector).  Forces,
potentials (dU/dq) and the k-space energy; rel-L2 <= 1e-5 (FP64) / 1e-4 (FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300.synthetic import positions_charges, random_kbatch

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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("P", [600, 2501])
def test_large_batch_matches_explicit_images(P, precision):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    Lx, Ly, H, gt, gb, M = 12.0, 9.0, 3.0, -0.7, 0.45, 6
    N = 777
    pos, q = positions_charges(N, Lx, Ly, H, seed=57)
    m = RBE2D(Lx, Ly, H, n_max=N, P=P, gamma_top=gt, gamma_bot=gb, M=M, Lz=-1, alpha=0.9, precision=precision)
    d = m.derived
    s = O.System(Lx=Lx, Ly=Ly, H=H, Lz=d["Lz"], gamma_top=gt, gamma_bot=gb, alpha=d["alpha"], M=d["M"])
    k = random_kbatch(P, nmax=(9, 8, 60), seed=P)
    m.set_k(k)
    F, phi, e = m.force(torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"), energy=True,
                        potential=True)
    ref = O.rbe(s, pos, q, k, mode=0, want_dq=True)
    eF = rel_l2(F.cpu().numpy(), ref["force"])
    eP = rel_l2(phi.cpu().numpy(), ref["dUdq"])
    print(f"P = {P} {precision}: force rel-L2 {eF:.2e}, dU/dq {eP:.2e}")
    assert eF < TOL[precision] and eP < TOL[precision]
    assert e.cpu().numpy()[0] == pytest.approx(ref["energy"][0], rel=TOL[precision])
    # the force without potential (the other kernel variant) on the same batch
    F2 = m.force(torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"))
    assert rel_l2(F2.cpu().numpy(), ref["force"]) < TOL[precision]
    m.sync_status()
    m.close()
