"""Host-side argument checks of the torch wrapper (paper_2405_06333_gb300/rbe2d.py).

The kernels read the wrapper's tensors as device memory of the context's GPU, so a host
tensor, a tensor on another device, a wrong shape or a wrong output buffer must be
refused before any call reaches the library.  The checks run on the CPU: the object is
built without a context, and every case here raises before the binding is called.
"""
import pytest
import torch

from paper_2405_06333_gb300.rbe2d import RBE2D


def _unbound(out_dtype=torch.float32):
    m = RBE2D.__new__(RBE2D)  # no context: only the checks are exercised
    m.device = torch.device("cuda", 0)
    m.out_dtype = out_dtype
    m.ctx = None
    return m


def test_host_tensors_are_refused():
    m = _unbound()
    with pytest.raises(ValueError, match="must be tensors on cuda:0"):
        m._inputs(torch.zeros((4, 3), dtype=torch.float64), torch.zeros(4, dtype=torch.float64))


def test_tensors_on_another_device_are_refused():
    m = _unbound()
    m.device = torch.device("cuda", 1)
    pos = torch.zeros((4, 3), dtype=torch.float64, device="meta")
    with pytest.raises(ValueError, match="must be tensors on cuda:1"):
        m._inputs(pos, torch.zeros(4, dtype=torch.float64, device="meta"))


def test_output_buffers_are_checked():
    m = _unbound(torch.float32)
    with pytest.raises(ValueError, match="out must be"):
        m._out(torch.zeros((4, 3), dtype=torch.float32), 4)  # host memory
    m.device = torch.device("meta")  # a device that needs no GPU, to reach the other checks
    ok = torch.empty((4, 3), dtype=torch.float32, device="meta")
    assert m._out(ok, 4) is ok
    for bad in (torch.empty((4, 3), dtype=torch.float64, device="meta"),   # precision
                torch.empty((5, 3), dtype=torch.float32, device="meta"),   # length
                torch.empty((3, 4), dtype=torch.float32, device="meta").t()):  # not contiguous
        with pytest.raises(ValueError, match="out must be"):
            m._out(bad, 4)


def test_shapes_are_checked():
    m = _unbound()
    m.device = torch.device("meta")
    pos = torch.empty((4, 3), dtype=torch.float64, device="meta")
    with pytest.raises(ValueError, match="pos must be"):
        m._inputs(pos, torch.empty(5, dtype=torch.float64, device="meta"))
    with pytest.raises(ValueError, match="pos must be"):
        m._inputs(torch.empty((4, 2), dtype=torch.float64, device="meta"),
                  torch.empty(4, dtype=torch.float64, device="meta"))
    p, q, flags = m._inputs(pos, torch.empty(4, dtype=torch.float64, device="meta"))
    assert p.shape == (4, 3) and q.shape == (4,) and flags == 0
