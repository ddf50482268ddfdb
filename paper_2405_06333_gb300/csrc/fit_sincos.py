"""Minimax fits of sin and cos on [-pi, pi] for the FMA-pipe sin/cos of the kernels.

sin x ~ x (s0 + s1 x^2 + ... + s5 x^10) and cos x ~ c0 + c1 x^2 + ... + c6 x^12 over the
whole circle, so that a kernel evaluates them on the radian argument it already has,
with no quadrant reduction (fused multiply-adds only).  Fitted by the Remez exchange
algorithm on the absolute error (in float64 with numpy), then rounded to float32.
Running this file prints the float32 constants that phase.cuh uses and their maximum
error evaluated in float64.
"""
import numpy as np


def remez(f, basis, lo, hi, n_iter=30, weight=None):
    """Minimax coefficients c of sum_k c_k basis_k(t) ~ f(t) on [lo, hi]."""
    m = len(basis)
    weight = weight or (lambda t: np.ones_like(t))
    # Chebyshev extrema as the starting reference (m + 1 points)
    k = np.arange(m + 1)
    ref = (lo + hi) / 2 + (hi - lo) / 2 * np.cos(np.pi * k / m)[::-1]
    grid = np.linspace(lo, hi, 200001)
    for _ in range(n_iter):
        A = np.zeros((m + 1, m + 1))
        for j, b in enumerate(basis):
            A[:, j] = b(ref)
        A[:, m] = (-1.0) ** np.arange(m + 1) / weight(ref)
        sol = np.linalg.solve(A, f(ref))
        c = sol[:m]
        err = (f(grid) - sum(cj * b(grid) for cj, b in zip(c, basis))) * weight(grid)
        # new reference: one extremum per sign run
        s = np.sign(err)
        s[s == 0] = 1
        idx = []
        start = 0
        for i in range(1, len(grid) + 1):
            if i == len(grid) or s[i] != s[start]:
                seg = np.arange(start, i)
                idx.append(seg[np.argmax(np.abs(err[seg]))])
                start = i
        idx = np.array(idx)
        while len(idx) > m + 1:  # drop the smallest end extremum
            if abs(err[idx[0]]) < abs(err[idx[-1]]):
                idx = idx[1:]
            else:
                idx = idx[:-1]
        if len(idx) == m + 1:
            ref = grid[idx]
    return c, np.max(np.abs(err))


def fit():
    h = np.pi
    # sin(x) = x (sin(x)/x): sin(x)/x as a polynomial in y = x^2 on [0, h^2], weighted by
    # |x| = sqrt(y) so that the absolute error of sin is minimised
    sc, _ = remez(lambda y: np.where(y > 0, np.sin(np.sqrt(y)) / np.sqrt(np.maximum(y, 1e-300)), 1.0),
                  [lambda y, p=p: y ** p for p in range(6)], 0.0, h * h,
                  weight=lambda y: np.sqrt(np.maximum(y, 1e-12)))
    cc, _ = remez(lambda y: np.cos(np.sqrt(y)), [lambda y, p=p: y ** p for p in range(7)], 0.0, h * h)
    s32 = np.asarray(sc, dtype=np.float32)
    c32 = np.asarray(cc, dtype=np.float32)
    x = np.linspace(-h, h, 400001)
    y = x * x
    sin_p = x * np.polyval(s32[::-1].astype(np.float64), y)
    cos_p = np.polyval(c32[::-1].astype(np.float64), y)
    return s32, c32, float(np.max(np.abs(sin_p - np.sin(x)))), float(np.max(np.abs(cos_p - np.cos(x))))


if __name__ == "__main__":
    s32, c32, es, ec = fit()
    print("sin:", ", ".join(f"{v:.9e}f" for v in s32), f"max abs err {es:.3e}")
    print("cos:", ", ".join(f"{v:.9e}f" for v in c32), f"max abs err {ec:.3e}")
