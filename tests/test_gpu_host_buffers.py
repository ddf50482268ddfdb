"""GPU checks of RBE2D_HOST_BUFFERS with pinned host memory, which the kernels read and
write in place (no staging copies): the same kernels see the same values, so forces,
potentials and energies equal those of the device-buffer call and of the staged call
with pageable host memory bit for bit, in both precisions and with the real-space part."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import positions_charges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


@pytest.mark.parametrize("precision,real,f32_in", [(B.RBE2D_FP32_MIXED, False, False), (B.RBE2D_FP32_MIXED, True, False),
                                                   (B.RBE2D_FP32_MIXED, False, True), (B.RBE2D_FP64, True, False)])
def test_pinned_host_buffers_equal_device_buffers(precision, real, f32_in):
    Lx, Ly, H, N = 40.0, 36.0, 6.0, 30011
    pos, q = positions_charges(N, Lx, Ly, H, seed=23)
    if f32_in:
        pos, q = pos.astype(np.float32), q.astype(np.float32)
    p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=-1, gamma_top=0.6, gamma_bot=-0.8, M=8, alpha=1.0, r_c=3.0, P=128,
                       seed=2, eps=1e-4, precision=precision, coulomb_k=1.0, real_space=1 if real else 0)
    ctx = B.rbe2d_init(p, N, torch.cuda.current_stream())
    B.rbe2d_sample_k(ctx, 3, None)
    odt = torch.float32 if precision == B.RBE2D_FP32_MIXED else torch.float64
    fl = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY | B.RBE2D_POTENTIAL
    fl |= (B.RBE2D_REAL if real else 0) | (B.RBE2D_INPUT_F32 if f32_in else 0)
    Fd = torch.empty((N, 3), dtype=odt, device="cuda")
    Pd = torch.empty(N, dtype=odt, device="cuda")
    Ed = torch.zeros(4, dtype=torch.float64, device="cuda")
    B.rbe2d_force(ctx, N, torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"), fl, Fd, Pd, Ed)
    torch.cuda.synchronize()
    results = {}
    for kind in ("pinned", "pageable"):
        mk = (lambda t: t.pin_memory()) if kind == "pinned" else (lambda t: t)
        hp, hq = mk(torch.as_tensor(pos).clone()), mk(torch.as_tensor(q).clone())
        for rep in range(2):
            Fh = mk(torch.full((N, 3), float("nan"), dtype=odt))
            Ph = mk(torch.full((N,), float("nan"), dtype=odt))
            Eh = mk(torch.zeros(4, dtype=torch.float64))
            B.rbe2d_force(ctx, N, hp, hq, fl | B.RBE2D_HOST_BUFFERS, Fh, Ph, Eh)
            results[(kind, rep)] = (Fh, Ph, Eh)
    for key, (Fh, Ph, Eh) in results.items():
        assert torch.equal(Fh, Fd.cpu()), key
        assert torch.equal(Ph, Pd.cpu()), key
        assert torch.equal(Eh, Ed.cpu()), key
    B.rbe2d_destroy(ctx)


@pytest.mark.parametrize("f32_in", [False, True])
@pytest.mark.parametrize("N", [1, 7, 17, 50, 113, 300])
def test_pinned_host_buffers_small_n(N, f32_in):
    """Host inputs read in place stage the first tile of each chunk in pieces of 16, 32
    and 64 particles and the rest: chunks shorter than a tile leave pieces empty or
    ragged (one chunk of 1, 7, 17, 50 or 113 particles; two of 150).  Same bits as the
    device-buffer call."""
    Lx, Ly, H = 9.0, 8.0, 3.0
    pos, q = positions_charges(N, Lx, Ly, H, seed=40 + N)  # neutral: odd N has one uncharged particle
    if f32_in:
        pos, q = pos.astype(np.float32), q.astype(np.float32)
    p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=-1, gamma_top=0.5, gamma_bot=-0.7, M=6, alpha=1.0, r_c=3.0, P=64,
                       seed=4, eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=0)
    ctx = B.rbe2d_init(p, N, torch.cuda.current_stream())
    B.rbe2d_sample_k(ctx, 1, None)
    fl = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY | B.RBE2D_POTENTIAL | (B.RBE2D_INPUT_F32 if f32_in else 0)
    Fd = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    Pd = torch.empty(N, dtype=torch.float32, device="cuda")
    Ed = torch.zeros(4, dtype=torch.float64, device="cuda")
    B.rbe2d_force(ctx, N, torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"), fl, Fd, Pd, Ed)
    torch.cuda.synchronize()
    hp, hq = torch.as_tensor(pos).clone().pin_memory(), torch.as_tensor(q).clone().pin_memory()
    Fh = torch.full((N, 3), float("nan"), dtype=torch.float32).pin_memory()
    Ph = torch.full((N,), float("nan"), dtype=torch.float32).pin_memory()
    Eh = torch.zeros(4, dtype=torch.float64).pin_memory()
    B.rbe2d_force(ctx, N, hp, hq, fl | B.RBE2D_HOST_BUFFERS, Fh, Ph, Eh)
    assert torch.equal(Fh, Fd.cpu())
    assert torch.equal(Ph, Pd.cpu())
    assert torch.equal(Eh, Ed.cpu())
    assert torch.isfinite(Fh).all()
    B.rbe2d_destroy(ctx)
