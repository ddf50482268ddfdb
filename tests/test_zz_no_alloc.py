"""The allocation-free structure-factor entry point (rbe2d_structure_factor_noalloc).

It serves callers that cannot allocate device memory on their call path (code inside
a global-mode stream capture, hosts whose device memory belongs to their own pool):
no context, and a fixed scratch array inside the library instead of cudaMalloc.  Its
results must equal those of the context-based rbe2d_structure_factor within the
structure-factor tolerance used by the other GPU tests (|d rho| <= 1e-6 sum|q| in the
float32-phase mode), on two calls in a row that share the scratch array.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


def _context_result(Lx, Ly, H, Lz, pos, q, k):
    from paper_2405_06333_gb300.rbe2d import RBE2D
    m = RBE2D(Lx, Ly, H, n_max=len(q), P=len(k), gamma_top=0.5, gamma_bot=-0.5, M=4, Lz=Lz, alpha=1.0,
              precision="fp32")
    m.set_k(k)
    out = m.structure_factor(torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"))
    torch.cuda.synchronize()
    m.close()
    return out.cpu().numpy()


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.synthetic import positions_charges, random_kbatch
    cases = [
        (40.0, 40.0, 5.0, 164.0, 10007, 200, 1),   # ragged N, part of the scratch used
        (30.0, 20.0, 4.0, 90.0, 4096, 512, 2),     # the largest batch the scratch holds
    ]
    for Lx, Ly, H, Lz, N, P, seed in cases:
        pos, q = positions_charges(N, Lx, Ly, H, seed=seed)
        k = random_kbatch(P, nmax=(10, 10, 60), seed=seed)
        out = torch.full((P, 4), float("nan"), dtype=torch.float64, device="cuda")
        B.rbe2d_structure_factor_noalloc(Lx, Ly, Lz, N, torch.as_tensor(pos, device="cuda"),
                                         torch.as_tensor(q, device="cuda"), P,
                                         torch.as_tensor(k, device="cuda"), out,
                                         torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _context_result(Lx, Ly, H, Lz, pos, q, k)
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref).max() / np.sum(np.abs(q))
        assert err < 1e-6, (N, P, err)


def test_noalloc_rejects_a_batch_larger_than_its_scratch():
    from paper_2405_06333_gb300 import binding as B
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(4, dtype=torch.float64, device="cuda")
    k = torch.ones((513, 3), dtype=torch.int32, device="cuda")
    out = torch.zeros((513, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RBE2DError) as ei:
        B.rbe2d_structure_factor_noalloc(10.0, 10.0, 30.0, 4, pos, q, 513, k, out)
    assert ei.value.code == B.RBE2D_EINVAL
