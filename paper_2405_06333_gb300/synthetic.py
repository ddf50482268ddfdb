"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws positions and charges
and names the workloads.  Charges are +1 for the first N/2 particles and -1 for the
rest (a neutral 1:1 electrolyte); positions are uniform in [0,Lx) x [0,Ly) x [0,H],
drawn in FP64 with numpy's PCG64 from a fixed seed, so charge sign is random in space.
The paper's own workloads (SPC/E water, LAMMPS electrolyte inputs) are not available;
these stand in for them with the same geometry, charge mix and particle counts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    Lx: float
    Ly: float
    H: float
    gamma_top: float
    gamma_bot: float
    M: int            # image levels; -1 = the Eq. 3.10 rule at eps
    alpha: float      # <= 0: the (N/(Lx Ly H))^(1/3) rule
    r_c: float        # <= 0: 3 / alpha
    Lz: float         # <= 0: the Eq. 3.23 rule at eps, rounded up
    P: int
    seed: int = 0     # k-batch Philox key
    pos_seed: int = 1
    eps: float = 1e-4


# The five workloads of the build, by geometry and size.
WORKLOADS = {
    "plain_n1e3": Workload("plain_n1e3", 1000, 20.0, 20.0, 10.0, 0.0, 0.0, 0, 0.5, 6.0, 40.0, 100),
    "dielectric_n1e4": Workload("dielectric_n1e4", 10000, 40.0, 40.0, 5.0, -0.95, -0.95, 20, 0.3, 8.0,
                                164.0, 200),
    "slab_n1e6": Workload("slab_n1e6", 1000000, 200.0, 200.0, 20.0, 0.9, -0.9, 14, 1.0772173450159417,
                          2.785, 594.0, 500),
    "thin_n1e6": Workload("thin_n1e6", 1000000, 200.0, 200.0, 2.0, 0.9, -0.9, 55, 2.3207944168063896,
                          1.293, 406.0, 500),
    "adjoint_n1e5": Workload("adjoint_n1e5", 100000, 100.0, 100.0, 10.0, -0.5, 0.8, 9, 1.0, 3.0, 247.0,
                             300),
}


def positions_charges(N: int, Lx: float, Ly: float, H: float, seed: int = 1):
    """N positions (N,3) float64 uniform in the slab and charges (N,) = +1 then -1."""
    rng = np.random.default_rng(seed)
    pos = np.empty((N, 3), dtype=np.float64)
    pos[:, 0] = rng.uniform(0.0, Lx, N)
    pos[:, 1] = rng.uniform(0.0, Ly, N)
    pos[:, 2] = rng.uniform(0.0, H, N)
    q = np.ones(N, dtype=np.float64)
    q[N // 2:] = -1.0
    if N % 2 == 1:
        q[-1] = 0.0
    return pos, q


def workload_inputs(w: Workload):
    return positions_charges(w.N, w.Lx, w.Ly, w.H, w.pos_seed)


def batched_systems(n_sys: int = 512, seed: int = 2, n_lo: int = 200, n_hi: int = 20000):
    """Independent slab systems of uneven size: N ~ U[n_lo, n_hi] (even), Lx = Ly ~ U[10, 60],
    H ~ U[1, 20], gamma_top, gamma_bot ~ U[-1, 1].  Returns a list of dicts with the
    geometry and the per-system position seed."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_sys):
        N = int(rng.integers(n_lo // 2, n_hi // 2 + 1)) * 2
        L = float(rng.uniform(10.0, 60.0))
        H = float(rng.uniform(1.0, 20.0))
        gt = float(rng.uniform(-1.0, 1.0))
        gb = float(rng.uniform(-1.0, 1.0))
        out.append({"N": N, "Lx": L, "Ly": L, "H": H, "gamma_top": gt, "gamma_bot": gb,
                    "pos_seed": 1000 + s})
    return out


def random_kbatch(P: int, nmax=(8, 8, 30), seed: int = 7):
    """A k-batch of P nonzero integer triples drawn uniformly in a box (not the method's
    sampler): used to test the force path independently of sampling."""
    rng = np.random.default_rng(seed)
    out = np.zeros((P, 3), dtype=np.int32)
    i = 0
    while i < P:
        n = rng.integers(-np.asarray(nmax), np.asarray(nmax) + 1)
        if np.any(n != 0):
            out[i] = n
            i += 1
    return out


def lattice_positions_charges(N: int, Lx: float, Ly: float, H: float, margin: float, seed: int = 1,
                              jitter: float = 0.1):
    """N charges on a jittered simple-cubic lattice filling [0,Lx)x[0,Ly)x[margin,H-margin]
    (no two closer than (1 - 2 jitter) times the spacing), charges +1/-1 in random order;
    a start for MD with repulsive cores."""
    rng = np.random.default_rng(seed)
    Hm = H - 2.0 * margin
    a = (Lx * Ly * Hm / N) ** (1.0 / 3.0)
    nx, ny = max(1, int(Lx / a)), max(1, int(Ly / a))
    nz = max(1, int(np.ceil(N / (nx * ny))))
    while nx * ny * nz < N:
        nz += 1
    ax, ay, az = Lx / nx, Ly / ny, Hm / nz
    idx = rng.permutation(nx * ny * nz)[:N]
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    pos = np.empty((N, 3))
    pos[:, 0] = (ix + 0.5 + jitter * rng.uniform(-1, 1, N)) * ax
    pos[:, 1] = (iy + 0.5 + jitter * rng.uniform(-1, 1, N)) * ay
    pos[:, 2] = margin + (iz + 0.5 + jitter * rng.uniform(-1, 1, N)) * az
    q = np.ones(N)
    q[N // 2:] = -1.0
    if N % 2 == 1:
        q[-1] = 0.0
    q = q[rng.permutation(N)]
    return pos, q


def random_positions_min_distance(N: int, Lx: float, Ly: float, H: float, d_min: float, margin: float = 0.0,
                                  seed: int = 1, max_tries: int = 100):
    """N positions uniform in [0,Lx) x [0,Ly) x [margin, H-margin], no two closer than d_min
    (x, y periodic), by random sequential placement on a grid of d_min cells; charges +1
    for a random half and -1 for the rest.  A disordered start for MD with repulsive cores
    (a lattice start carries its order into the first configurations)."""
    rng = np.random.default_rng(seed)
    nc = [max(1, int(Lx / d_min)), max(1, int(Ly / d_min)), max(1, int((H - 2 * margin) / d_min))]
    cs = [Lx / nc[0], Ly / nc[1], (H - 2 * margin) / nc[2]]
    grid = {}
    pos = np.empty((N, 3))
    n = 0
    while n < N:
        for _ in range(max_tries):
            p = np.array([rng.uniform(0, Lx), rng.uniform(0, Ly), rng.uniform(margin, H - margin)])
            c = [min(int(p[0] / cs[0]), nc[0] - 1), min(int(p[1] / cs[1]), nc[1] - 1),
                 min(int((p[2] - margin) / cs[2]), nc[2] - 1)]
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        key = ((c[0] + dx) % nc[0], (c[1] + dy) % nc[1], c[2] + dz)
                        for j in grid.get(key, ()):
                            d = pos[j] - p
                            d[0] -= Lx * round(d[0] / Lx)
                            d[1] -= Ly * round(d[1] / Ly)
                            if d @ d < d_min * d_min:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[n] = p
                grid.setdefault((c[0], c[1], c[2]), []).append(n)
                n += 1
                break
        else:
            raise RuntimeError("random_positions_min_distance: density too high for d_min")
    q = np.ones(N)
    q[N // 2:] = -1.0
    if N % 2 == 1:
        q[-1] = 0.0
    return pos, q[rng.permutation(N)]
