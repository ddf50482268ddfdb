"""The FMA-pipe sin/cos polynomials: the constants in the kernel are the ones
csrc/fit_sincos.py derives by the Remez exchange, and their error on [-pi/4, pi/4]
stays below 5e-9 (evaluated in float64) and below 2e-7 when evaluated in float32 over
the whole circle with the kernel's quadrant reduction of a 32-bit turn."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fit():
    import importlib.util
    spec = importlib.util.spec_from_file_location("fit", os.path.join(ROOT, "paper_2405_06333_gb300", "csrc",
                                                                      "fit_sincos.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m.fit()


def _kernel_constants():
    src = open(os.path.join(ROOT, "paper_2405_06333_gb300", "csrc", "phase.cuh")).read()
    body = src[src.index("void sincos_poly32"):]
    body = body[:body.index("}")]
    return [float(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]


def test_fit_error_bounds_and_kernel_constants():
    s32, c32, es, ec = _fit()
    assert es < 5e-9 and ec < 5e-9
    consts = _kernel_constants()
    want = [s32[3], s32[2], s32[1], c32[4], c32[3], c32[2]]
    assert len(consts) >= 6
    np.testing.assert_array_equal(np.float32(consts[-6:]), np.float32(want))


def test_float32_evaluation_with_quadrant_reduction():
    s32, c32, _, _ = _fit()
    rng = np.random.default_rng(0)
    t = np.concatenate([rng.integers(0, 2**32, 200000, dtype=np.uint64),
                        np.array([0, 2**29, 2**29 - 1, 2**30, 2**31, 2**32 - 1, 3 * 2**30 - 1], dtype=np.uint64)])
    t = t.astype(np.uint32)
    qd = ((t.astype(np.uint64) + 0x20000000) >> 30).astype(np.uint32) & 3
    r = (t.astype(np.int64) - (qd.astype(np.int64) << 30))
    r = ((r + 2**31) % 2**32 - 2**31).astype(np.int32)
    x = np.float32(r) * np.float32(1.46291807926715968e-09)
    y = np.float32(x * x)
    f = np.float32
    sp = x * f(f(f(f(s32[3]) * y + f(s32[2])) * y + f(s32[1])) * y + f(1.0))
    cp = f(f(f(f(f(c32[4]) * y + f(c32[3])) * y + f(c32[2])) * y + f(-0.5)) * y + f(1.0))
    odd = (qd & 1) == 1
    ss, cc = np.where(odd, cp, sp), np.where(odd, sp, cp)
    s = np.where(qd & 2, -ss, ss)
    c = np.where((qd + 1) & 2, -cc, cc)
    ang = 2 * np.pi * t.astype(np.float64) / 2**32
    assert np.max(np.abs(s - np.sin(ang))) < 2e-7
    assert np.max(np.abs(c - np.cos(ang))) < 2e-7
