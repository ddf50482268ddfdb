"""The allocation-free structure-factor entry point (rbe2d_structure_factor_noalloc).

It serves callers that cannot allocate device memory on their call path (code inside
a global-mode stream capture, hosts whose device memory belongs to their own pool):
no context, and a fixed scratch array inside the library instead of cudaMalloc.  Its
results must equal those of the context-based rbe2d_structure_factor and the FP64
oracle's rho and sigma within the structure-factor tolerance used by the other GPU
tests (|d rho| <= 1e-6 sum|q| in the float32-phase mode), on calls in a row that share
the scratch array, including a small call after a full one (most particle chunks then
empty) and a call without particles (all sums zero).

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


def _noalloc(B, Lx, Ly, Lz, pos, q, k):
    N, P = len(q), len(k)
    out = torch.full((P, 4), float("nan"), dtype=torch.float64, device="cuda")
    pd = torch.as_tensor(pos, device="cuda").reshape(N, 3)
    qd = torch.as_tensor(q, device="cuda")
    B.rbe2d_structure_factor_noalloc(Lx, Ly, Lz, N, pd, qd, P, torch.as_tensor(k, device="cuda"), out,
                                     torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    import oracle as O
    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.synthetic import positions_charges, random_kbatch
    cases = [
        (40.0, 40.0, 5.0, 164.0, 10007, 200, 1),   # ragged N, part of the scratch used
        (30.0, 20.0, 4.0, 90.0, 4096, 512, 2),     # the largest batch the scratch holds
        (25.0, 25.0, 3.0, 80.0, 100, 37, 3),       # most particle chunks empty after a full call
        (35.0, 35.0, 4.0, 100.0, 3001, 300, 5),    # 3 wave-vector slots per thread
    ]
    for Lx, Ly, H, Lz, N, P, seed in cases:
        pos, q = positions_charges(N, Lx, Ly, H, seed=seed)
        k = random_kbatch(P, nmax=(10, 10, 60), seed=seed)
        got = _noalloc(B, Lx, Ly, Lz, pos, q, k)
        ref = _context_result(Lx, Ly, H, Lz, pos, q, k)
        assert np.all(np.isfinite(got))
        l1 = np.sum(np.abs(q))
        err = np.abs(got - ref).max() / l1
        assert err < 1e-6, (N, P, err)
        # and against the FP64 oracle's rho and sigma directly (Eq. 3.17, Sec. 3.4)
        s = O.System(Lx=Lx, Ly=Ly, H=H, Lz=Lz, gamma_top=0.5, gamma_bot=-0.5, alpha=1.0, M=4)
        err_o = np.abs(got - O.rho_sigma(s, pos, q, k)).max() / l1
        assert err_o < 1e-6, (N, P, err_o)
    # no particles after calls that left partial sums in the scratch: every sum is zero
    k = random_kbatch(64, nmax=(10, 10, 60), seed=4)
    got = _noalloc(B, 10.0, 10.0, 30.0, np.zeros((0, 3)), np.zeros(0), k)
    assert np.array_equal(got, np.zeros((64, 4)))


def test_noalloc_rejects_a_batch_larger_than_its_scratch():
    from paper_2405_06333_gb300 import binding as B
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(4, dtype=torch.float64, device="cuda")
    k = torch.ones((513, 3), dtype=torch.int32, device="cuda")
    out = torch.zeros((513, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RBE2DError) as ei:
        B.rbe2d_structure_factor_noalloc(10.0, 10.0, 30.0, 4, pos, q, 513, k, out)
    assert ei.value.code == B.RBE2D_EINVAL
