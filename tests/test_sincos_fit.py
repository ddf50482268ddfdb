"""The FMA-pipe sin/cos polynomials: the constants in the kernels are the ones
csrc/fit_sincos.py derives by the Remez exchange; their error over the whole circle
stays below 2.5e-7 (evaluated in float64), and below 5e-7 against the sine and cosine of
the float32 radian argument when evaluated the way the kernels do (float32 fused
multiply-adds on (float)(int32)t x 2 pi / 2^32)."""
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


def _kernel_constants(name):
    src = open(os.path.join(ROOT, "paper_2405_06333_gb300", "csrc", "phase.cuh")).read()
    body = re.search(r"#define " + name + r"(.*?)\n(?:#define|__device__)", src, re.S).group(1)
    return [float(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]


def _fma_f32(a, b, c):
    """float32 fused multiply-add: the exact a b + c (float64 holds the product of two
    float32 exactly) rounded once to float32."""
    return np.float32(a.astype(np.float64) * b.astype(np.float64) + np.float64(c))


def _eval_f32(s32, c32, x):
    y = np.float32(x * x)
    p = np.full_like(x, s32[-1])
    for cf in s32[-2::-1]:
        p = _fma_f32(p, y, cf)
    q = np.full_like(x, c32[-1])
    for cf in c32[-2::-1]:
        q = _fma_f32(q, y, cf)
    return np.float32(x * p), q


def test_fit_error_bounds_and_kernel_constants():
    s32, c32, es, ec = _fit()
    assert es < 2.5e-7 and ec < 1e-7
    np.testing.assert_array_equal(np.float32(_kernel_constants("RBE2D_SIN_POLY")), s32)
    np.testing.assert_array_equal(np.float32(_kernel_constants("RBE2D_COS_POLY")), c32)
    # the series it approximates: leading terms of the Taylor series of sin and cos
    assert abs(s32[0] - 1) < 1e-6 and abs(s32[1] + 1 / 6) < 1e-5
    assert c32[0] == 1 and abs(c32[1] + 0.5) < 1e-6


def test_float32_evaluation_over_the_circle():
    s32, c32, _, _ = _fit()
    rng = np.random.default_rng(0)
    t = np.concatenate([rng.integers(0, 2**32, 400000, dtype=np.uint64),
                        np.array([0, 1, 2**29, 2**30, 2**31 - 1, 2**31, 2**31 + 1, 3 * 2**30, 2**32 - 1],
                                 dtype=np.uint64)]).astype(np.uint32)
    x = np.float32(t.view(np.int32)) * np.float32(1.46291807926715968e-09)
    s, c = _eval_f32(s32, c32, x)
    xd = x.astype(np.float64)
    assert np.max(np.abs(s - np.sin(xd))) < 5e-7
    assert np.max(np.abs(c - np.cos(xd))) < 5e-7
    # the end points of the circle: sin(+-pi) ~ 0, cos(+-pi) ~ -1
    end = np.float32([-np.pi, np.pi])
    se, ce = _eval_f32(s32, c32, end)
    assert np.all(np.abs(se) < 5e-7) and np.all(np.abs(ce + 1) < 5e-7)
