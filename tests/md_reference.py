"""Host reference of one Langevin MD step, written for the MD tests (numpy, float64).

It restates, independently of the CUDA kernels, what one step of the library's MD loop
computes (the Langevin equation of Sec. 2.4 integrated by the BAOAB splitting of
Leimkuhler and Matthews, 2013):
  B  v <- v + (dt/2m) F(x)            F: the pair/k-space force plus the walls at x
  A  x <- x + (dt/2) v
  O  v <- c1 v + sqrt(1 - c1^2) sqrt(kT/m) xi,   c1 = exp(-gamma dt)
  A  x <- x + (dt/2) v,  then x, y wrapped into the cell
  B  v <- v + (dt/2m) F(x')           with the force at the new positions
The walls at z = 0 and z = H are the purely repulsive shifted Lennard-Jones (WCA) walls
of the paper's electrolyte test (Sec. 4.1):
  F(d) = 24 eps [2 (sigma/d)^12 - (sigma/d)^6] / d  for d < 2^(1/6) sigma, else 0,
pushing away from the wall, with d the distance to it; the library evaluates it no
closer than d = sigma/2 (its stated cap).
The normals xi come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
(i mod 2^32, i >> 32, step mod 2^32, step >> 32) and key (seed mod 2^32, seed >> 32),
through the Box-Muller transform of the four words w0..w3 as the library documents it:
u1 = ((w0 >> 8) + 1/2) 2^-24, u2 = (w1 >> 8) 2^-24, u3, u4 likewise from w2, w3, the
sum formed in float32 (so 2^24 - 1/2 rounds to 2^24 and u1 can be 1);
xi = (r1 cos 2 pi u2, r1 sin 2 pi u2, r3 cos 2 pi u4), r = sqrt(-2 ln u).
"""
from __future__ import annotations

import numpy as np

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """Philox4x32-10 of counters ctr (n x 4, uint32 values) under key (2 uint32 values):
    ten rounds of two 32 x 32 -> 64-bit products, the key bumped by the Weyl constants
    before every round after the first.  Returns n x 4 uint64 holding 32-bit words."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy()
    k0, k1 = np.uint64(int(key[0]) & 0xFFFFFFFF), np.uint64(int(key[1]) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> _S32) ^ c1 ^ k0), (p1 & _MASK), ((p0 >> _S32) ^ c3 ^ k1), (p0 & _MASK)
    return np.stack([c0, c1, c2, c3], axis=1)


def thermostat_normals(N, step, seed):
    """N x 3 standard normals of MD step `step` for particles 0..N-1."""
    i = np.arange(N, dtype=np.uint64)
    s = np.uint64(step)
    ctr = np.stack([i & _MASK, i >> _S32, np.full(N, s & _MASK), np.full(N, s >> _S32)], axis=1)
    w = philox4x32_10(ctr, (int(seed) & 0xFFFFFFFF, int(seed) >> 32))
    u = lambda x, half: ((x >> np.uint64(8)).astype(np.float32) + np.float32(0.5 if half else 0.0)).astype(
        np.float64) * 2.0 ** -24
    u1, u2, u3, u4 = u(w[:, 0], True), u(w[:, 1], False), u(w[:, 2], True), u(w[:, 3], False)
    r1, r3 = np.sqrt(-2.0 * np.log(u1)), np.sqrt(-2.0 * np.log(u3))
    return np.stack([r1 * np.cos(2 * np.pi * u2), r1 * np.sin(2 * np.pi * u2), r3 * np.cos(2 * np.pi * u4)], axis=1)


def wca_wall(d, sigma, eps):
    """Magnitude of the WCA wall force at distance d (positive: away from the wall)."""
    d = np.asarray(d, dtype=np.float64)
    if sigma <= 0:
        return np.zeros_like(d)
    dd = np.maximum(d, 0.5 * sigma)
    s6 = (sigma / dd) ** 6
    f = 24.0 * eps * (2.0 * s6 * s6 - s6) / dd
    return np.where(d < 2.0 ** (1.0 / 6.0) * sigma, f, 0.0)


def wall_force_z(z, H, sigma, eps):
    """z force of both walls on particles at heights z."""
    return wca_wall(z, sigma, eps) - wca_wall(H - z, sigma, eps)


def baoab_step(x, v, F0, F1, *, dt, gamma, kT, mass, H, Lx, Ly, sigma_wall=0.0, eps_wall=0.0, xi=None):
    """One BAOAB step from (x, v) with force F0 at x; F1 is the force (without walls) at
    the positions the step reaches (the caller evaluates it there).  Returns (x', v')."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    hk, h = 0.5 * dt / mass, 0.5 * dt
    c1 = np.exp(-gamma * dt)
    a0 = np.array(F0, dtype=np.float64)
    a0[:, 2] += wall_force_z(x[:, 2], H, sigma_wall, eps_wall)
    v = v + hk * a0
    x = x + h * v
    v = c1 * v
    if xi is not None:
        v = v + np.sqrt(max(0.0, 1.0 - c1 * c1)) * np.sqrt(kT / mass) * xi
    x = x + h * v
    x[:, 0] -= np.floor(x[:, 0] / Lx) * Lx
    x[:, 1] -= np.floor(x[:, 1] / Ly) * Ly
    a1 = np.array(F1, dtype=np.float64)
    a1[:, 2] += wall_force_z(x[:, 2], H, sigma_wall, eps_wall)
    v = v + hk * a1
    return x, v
