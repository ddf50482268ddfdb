"""CPU checks of the boundary: the library builds, loads without a GPU and exports
every entry point that include/rbe2d.h declares; the binding mirrors them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbe2d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbe2d_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_hot_path_entry_points():
    names = _declared()
    for n in ("rbe2d_init", "rbe2d_sample_k", "rbe2d_structure_factor", "rbe2d_force", "rbe2d_energy_backward"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2405_06333_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_has_same_names():
    from paper_2405_06333_gb300 import binding
    for n in _declared():
        assert hasattr(binding, n), n


def test_init_without_gpu_fails_cleanly_or_reports():
    """Without a GPU the context cannot be created; the call must return an error code
    (never crash), and the binding raises RBE2DError."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2405_06333_gb300 import binding as B
    B.lib()
    p = B.rbe2d_params(Lx=10, Ly=10, H=5, Lz=-1, gamma_top=0, gamma_bot=0, M=0, alpha=1.0, r_c=3.0, P=8, seed=0,
                       eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0)
    with pytest.raises(B.RBE2DError):
        B.rbe2d_init(p, 100, stream=0)


def test_init_rejects_bad_parameters_before_touching_the_device():
    from paper_2405_06333_gb300 import binding as B
    mk = lambda **kw: B.rbe2d_params(**{**dict(Lx=10, Ly=10, H=5, Lz=-1, gamma_top=0, gamma_bot=0, M=0, alpha=1.0,
                                               r_c=3.0, P=8, seed=0, eps=1e-4, precision=1, coulomb_k=1.0), **kw})
    for bad in (dict(gamma_top=1.5), dict(P=0), dict(Lx=-1.0), dict(M=4, gamma_top=0.5, Lz=10.0), dict(precision=7)):
        with pytest.raises(B.RBE2DError) as ei:
            B.rbe2d_init(mk(**bad), 100, stream=0)
        assert ei.value.code == B.RBE2D_EINVAL


def test_timer_entry_points_reject_a_null_context():
    from paper_2405_06333_gb300 import binding as B
    L = B.lib()
    assert L.rbe2d_timer_enable(None, 4, B.RBE2D_TIMER_ALL) == B.RBE2D_EINVAL
    assert L.rbe2d_timer_read(None, None, None) == B.RBE2D_EINVAL
    assert len(B.TIMER_NAMES) == B.RBE2D_TIMER_COUNT == 7


def test_kernel_launch_counter_needs_no_gpu():
    from paper_2405_06333_gb300 import binding as B
    L = B.lib()
    assert L.rbe2d_kernel_launches(None) == B.RBE2D_EINVAL
    assert B.rbe2d_kernel_launches() >= 0
