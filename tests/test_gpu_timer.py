"""GPU checks of the per-kernel timer (a measurement aid with no counterpart in the
paper): it records one event pair per launch of each kernel class, stops at its
capacity, skips graph capture, and its times add up to no more than the step time."""
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


def _ctx(N, precision):
    p = B.rbe2d_params(Lx=30.0, Ly=30.0, H=6.0, Lz=-1, gamma_top=0.7, gamma_bot=-0.3, M=6, alpha=0.9, r_c=3.5, P=64,
                       seed=3, eps=1e-4, precision=precision, coulomb_k=1.0, real_space=0)
    return B.rbe2d_init(p, N, torch.cuda.current_stream())


@pytest.mark.parametrize("precision", [B.RBE2D_FP32_MIXED, B.RBE2D_FP64])
def test_timer_counts_launches_and_stops_at_capacity(precision):
    N = 20000
    pos, q = positions_charges(N, 30.0, 30.0, 6.0, seed=5)
    pos, q = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    ctx = _ctx(N, precision)
    F = torch.empty((N, 3), dtype=torch.float32 if precision == B.RBE2D_FP32_MIXED else torch.float64, device="cuda")
    fl = B.RBE2D_KSPACE | B.RBE2D_IBC
    B.rbe2d_timer_enable(ctx, 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(3):
        B.rbe2d_sample_k(ctx, s, None)
        B.rbe2d_force(ctx, N, pos, q, fl, F)
    e1.record()
    t = B.rbe2d_timer_read(ctx)
    total = e0.elapsed_time(e1)
    for name in ("sample", "structure_factor", "fold", "force"):
        ms, n = t[name]
        assert n == 3 and ms > 0, (name, t[name])
    assert t["pack"][1] == (3 if precision == B.RBE2D_FP64 else 0)
    assert t["real_space"][1] == 0 and t["md"][1] == 0
    assert sum(ms for ms, _ in t.values()) <= total * 1.001 + 1e-3
    # records were cleared by the read; past the capacity nothing more is recorded
    for s in range(6):
        B.rbe2d_sample_k(ctx, s, None)
    t = B.rbe2d_timer_read(ctx)
    assert t["sample"][1] == 4 and t["force"][1] == 0
    # only the selected classes are recorded
    B.rbe2d_timer_enable(ctx, 4, ("force",))
    B.rbe2d_sample_k(ctx, 0, None)
    B.rbe2d_force(ctx, N, pos, q, fl, F)
    t = B.rbe2d_timer_read(ctx)
    assert t["force"][1] == 1 and t["sample"][1] == 0 and t["structure_factor"][1] == 0
    B.rbe2d_timer_enable(ctx, 0)
    B.rbe2d_sample_k(ctx, 0, None)
    assert B.rbe2d_timer_read(ctx)["sample"] == (0.0, 0)
    assert B.status_code(B.rbe2d_timer_enable, ctx, -1) == B.RBE2D_EINVAL
    B.rbe2d_destroy(ctx)


def test_timer_skips_graph_capture():
    N = 4096
    pos, q = positions_charges(N, 30.0, 30.0, 6.0, seed=6)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pos, q = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
        p = B.rbe2d_params(Lx=30.0, Ly=30.0, H=6.0, Lz=-1, gamma_top=0.7, gamma_bot=-0.3, M=6, alpha=0.9, r_c=3.5,
                           P=64, seed=3, eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=0)
        ctx = B.rbe2d_init(p, N, s)
        F = torch.empty((N, 3), device="cuda")
        step = torch.zeros(1, dtype=torch.int64, device="cuda")
        B.rbe2d_sample_k_dev(ctx, step, None)
        B.rbe2d_force(ctx, N, pos, q, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
        s.synchronize()
        B.rbe2d_timer_enable(ctx, 8)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            B.rbe2d_sample_k_dev(ctx, step, None)
            B.rbe2d_force(ctx, N, pos, q, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
        g.replay()
        t = B.rbe2d_timer_read(ctx)
        assert all(n == 0 for _, n in t.values()), t
        F1 = F.clone()
        B.rbe2d_force(ctx, N, pos, q, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
        t = B.rbe2d_timer_read(ctx)
        assert t["force"][1] == 1
        assert torch.equal(F, F1)
    B.rbe2d_destroy(ctx)


def test_kernel_launch_counter_counts_each_kernel():
    """One bench step (draw, structure factor with the fold, force reusing it) is four
    kernels in FP32-mixed mode and five in FP64 mode (separate packing)."""
    N = 5000
    pos, q = positions_charges(N, 30.0, 30.0, 6.0, seed=8)
    pos, q = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    for precision, per_step in ((B.RBE2D_FP32_MIXED, 4), (B.RBE2D_FP64, 5)):
        ctx = _ctx(N, precision)
        F = torch.empty((N, 3), dtype=torch.float32 if precision == B.RBE2D_FP32_MIXED else torch.float64,
                        device="cuda")
        n0 = B.rbe2d_kernel_launches()
        for s in range(3):
            B.rbe2d_sample_k(ctx, s, None)
            B.rbe2d_structure_factor(ctx, N, pos, q, 0, None)
            B.rbe2d_force(ctx, N, pos, q, B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REUSE_SF, F)
        assert B.rbe2d_kernel_launches() - n0 == 3 * per_step
        B.rbe2d_destroy(ctx)
