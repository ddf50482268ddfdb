"""Independent reference sums used to pin the oracle (test code, not the oracle).

- ``ewald2d_energy``: the exact quasi-2D Ewald sum (Eqs. 2.5-2.9, "Ewald2D") for a
  set of target charges in a doubly periodic cell interacting with a set of source
  charges.  The dielectric case feeds the image charges of Eq. 3.2 / Eq. 3.3 as extra
  sources (each image layer is neutral because the real charges are).  No k_z
  discretisation and no L_z enter, so it is a different route from the oracle's
  Ewald3D-plus-IBC sum (Theorem 2.1, Theorem 3.3).
- ``direct_energy``: a plain lattice sum over a disc of xy replicas, for the overall
  scale of ``ewald2d_energy`` in a large cell.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc, erfcx, erf


def _exp_erfc(h, z, alpha):
    """e^{h z} erfc(h/(2 alpha) + alpha z) without overflow."""
    a = h / (2.0 * alpha) + alpha * z
    g = np.exp(-h * h / (4.0 * alpha * alpha) - alpha * alpha * z * z)
    pos = erfcx(np.abs(a)) * g
    return np.where(a >= 0, pos, 2.0 * np.exp(h * z) - pos)


def image_sources(pos, q, H, gt, gb, M):
    """Real charges plus their images up to level M, with the physical coefficient
    convention: the first image above the slab (2H - z) is the reflection in the top
    interface and carries gamma_top; the first below (-z) carries gamma_bot.  Images
    are built by repeated reflection, not from the closed-form coefficient tables."""
    src_p = [pos.copy()]
    src_q = [q.copy()]
    # chains of reflections starting at the top (t) or the bottom (b) interface
    for start in ("t", "b"):
        z = pos[:, 2].copy()
        coef = np.ones_like(q)
        side = start
        for l in range(1, M + 1):
            if side == "t":
                z = 2.0 * H - z
                coef = coef * gt
                side = "b"
            else:
                z = -z
                coef = coef * gb
                side = "t"
            p = pos.copy()
            p[:, 2] = z
            src_p.append(p)
            src_q.append(q * coef)
    return np.concatenate(src_p), np.concatenate(src_q)


def ewald2d_energy(pos, q, src_pos, src_q, Lx, Ly, alpha, same_index=None, nrep=None, mmax=None):
    """U = 1/2 sum_i q_i sum_src q_src psi(r_i - r_src) - alpha/sqrt(pi) sum q_i^2.

    psi = real-space erfc lattice sum + Fourier part with G_alpha (Eq. 2.8) + the
    zero-mode term of Eq. 2.9.  same_index[i] is the source index of target i itself
    (its n = 0 real-space term is excluded)."""
    N = len(q)
    if nrep is None:
        nrep = int(np.ceil(7.0 / (alpha * min(Lx, Ly)))) + 1
    if mmax is None:
        hmax = 2.0 * alpha * np.sqrt(46.0) + 1.0
        mmax = (int(np.ceil(hmax * Lx / (2 * np.pi))), int(np.ceil(hmax * Ly / (2 * np.pi))))
    mx = np.arange(-mmax[0], mmax[0] + 1)
    my = np.arange(-mmax[1], mmax[1] + 1)
    MX, MY = np.meshgrid(mx, my, indexing="ij")
    keep = ~((MX == 0) & (MY == 0))
    hx = 2 * np.pi * MX[keep] / Lx
    hy = 2 * np.pi * MY[keep] / Ly
    h = np.sqrt(hx * hx + hy * hy)
    A = Lx * Ly
    U = 0.0
    for i in range(N):
        d = pos[i][None, :] - src_pos
        # real space
        ur = 0.0
        for nx in range(-nrep, nrep + 1):
            for ny in range(-nrep, nrep + 1):
                dx = d[:, 0] + nx * Lx
                dy = d[:, 1] + ny * Ly
                r = np.sqrt(dx * dx + dy * dy + d[:, 2] ** 2)
                if nx == 0 and ny == 0 and same_index is not None:
                    r = r.copy()
                    r[same_index[i]] = np.inf
                ur += np.sum(src_q * erfc(alpha * r) / r)
        # Fourier part
        z = d[:, 2]
        phase = np.cos(np.outer(hx, d[:, 0]) + np.outer(hy, d[:, 1]))
        G = _exp_erfc(h[:, None], z[None, :], alpha) + _exp_erfc(h[:, None], -z[None, :], alpha)
        uf = np.pi / A * np.sum(src_q[None, :] * phase * G / h[:, None])
        uj = -2.0 * np.pi / A * np.sum(src_q * (z * erf(alpha * z) + np.exp(-(alpha * z) ** 2) / (alpha * np.sqrt(np.pi))))
        U += 0.5 * q[i] * (ur + uf + uj)
    return U - alpha / np.sqrt(np.pi) * np.sum(q * q)


def dielectric_energy(pos, q, Lx, Ly, H, gt, gb, M, alpha):
    """Truncated image energy U^c_M (Eq. 3.2 summed to l = M) by the exact Ewald2D sum."""
    sp, sq = image_sources(pos, q, H, gt, gb, M)
    return ewald2d_energy(pos, q, sp, sq, Lx, Ly, alpha, same_index=np.arange(len(q)))


def direct_energy(pos, q, Lx, Ly, R):
    """1/2 sum' q_i q_j / |r_ij + l| over xy replicas with |l| <= R (no images)."""
    N = len(q)
    nr = int(np.ceil(R / min(Lx, Ly)))
    U = 0.0
    for nx in range(-nr, nr + 1):
        for ny in range(-nr, nr + 1):
            lx, ly = nx * Lx, ny * Ly
            if lx * lx + ly * ly > R * R:
                continue
            for i in range(N):
                d = pos[i] - pos + np.array([lx, ly, 0.0])
                r = np.sqrt(np.sum(d * d, axis=1))
                if nx == 0 and ny == 0:
                    r[i] = np.inf
                U += 0.5 * q[i] * np.sum(q / r)
    return U
