"""Python access to the FP64 CPU oracle (oracle/rbe2d_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py, never by the CUDA path.  Every function
here only marshals numpy arrays into the C oracle; the arithmetic lives in C and
follows the paper (arXiv 2405.06333) section by section, see the C file's header.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


class _OrcSystem(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("H", C.c_double), ("Lz", C.c_double),
                ("gamma_top", C.c_double), ("gamma_bot", C.c_double), ("alpha", C.c_double),
                ("M", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
        vp = C.c_void_p
        sysp = P(_OrcSystem)
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_set_num_threads.restype = None
        L.orc_philox4x64_10.argtypes = [vp, vp, vp]
        L.orc_nmax.argtypes = [d, d]; L.orc_nmax.restype = C.c_int
        L.orc_w1d.argtypes = [C.c_int, d, d]; L.orc_w1d.restype = d
        L.orc_S.argtypes = [sysp]; L.orc_S.restype = d
        L.orc_cdf.argtypes = [d, d, C.c_int, vp]
        L.orc_sample_k.argtypes = [sysp, u64, u64, C.c_int, vp]; L.orc_sample_k.restype = C.c_int
        L.orc_full_klist.argtypes = [sysp, vp, vp, vp]; L.orc_full_klist.restype = i64
        L.orc_metropolis.argtypes = [sysp, u64, u64, C.c_int, C.c_int, vp, vp]
        L.orc_metropolis_halfwidth.argtypes = [d, d]; L.orc_metropolis_halfwidth.restype = C.c_int
        L.orc_image_coeff.argtypes = [sysp, C.c_int, vp, vp, vp, vp, vp, vp]
        L.orc_image_z.argtypes = [sysp, C.c_int, d, vp, vp]
        L.orc_cM.argtypes = [sysp]; L.orc_cM.restype = d
        L.orc_Y.argtypes = [sysp, d, vp, vp]
        L.orc_dY.argtypes = [sysp, d, C.c_int, vp, vp]
        L.orc_sf_explicit.argtypes = [sysp, i64, vp, vp, i64, vp, vp, vp, vp, vp]
        L.orc_sf_recal.argtypes = [sysp, i64, vp, vp, i64, vp, vp, vp, vp]
        L.orc_kspace.argtypes = [sysp, i64, vp, vp, i64, vp, vp, C.c_int, i64, vp, vp, vp, vp, vp]
        L.orc_kspace.restype = C.c_int
        L.orc_rho_sigma.argtypes = [sysp, i64, vp, vp, i64, vp, vp]
        L.orc_real_space.argtypes = [sysp, d, i64, vp, vp, i64, vp, vp, vp]
        L.orc_real_space.restype = C.c_int
        L.orc_auto_M.argtypes = [d, d, d, d, d, d]; L.orc_auto_M.restype = C.c_int
        L.orc_auto_Lz.argtypes = [d, d, d, C.c_int, d, d]; L.orc_auto_Lz.restype = d
        L.orc_auto_alpha.argtypes = [i64, d, d, d]; L.orc_auto_alpha.restype = d
        _lib = L
    return _lib


@dataclass
class System:
    """Slab geometry and method parameters, in the paper's notation."""
    Lx: float
    Ly: float
    H: float
    Lz: float
    gamma_top: float = 0.0
    gamma_bot: float = 0.0
    alpha: float = 1.0
    M: int = 0

    def c(self):
        return _OrcSystem(self.Lx, self.Ly, self.H, self.Lz, self.gamma_top, self.gamma_bot,
                          self.alpha, int(self.M))

    @property
    def V(self):
        return self.Lx * self.Ly * self.Lz


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the OpenMP loops from now on (timing only: the per-k and per-particle
    sums do not depend on it; the real-space energy total may differ in its last bits)."""
    lib().orc_set_num_threads(int(n))


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def nmax(alpha, L):
    return lib().orc_nmax(alpha, L)


def w1d(n, alpha, L):
    return lib().orc_w1d(int(n), alpha, L)


def S(s: System) -> float:
    sc = s.c()
    return lib().orc_S(C.byref(sc))


def cdf(alpha, L):
    nd = nmax(alpha, L)
    out = np.zeros(2 * nd + 1)
    lib().orc_cdf(alpha, L, nd, _p(out))
    return out


def sample_k(s: System, seed: int, step: int, P: int) -> np.ndarray:
    sc = s.c()
    out = np.zeros((P, 3), dtype=np.int32)
    st = lib().orc_sample_k(C.byref(sc), seed, step, P, _p(out))
    if st != 0:
        raise RuntimeError("oracle sampler exhausted its attempts")
    return out


def metropolis(s: System, seed: int, step: int, sweeps: int, state):
    """Advance every chain of `state` (P x 3 int32) by `sweeps` Metropolis updates of
    step `step`; returns (new state, number of accepted moves)."""
    sc = s.c()
    st = np.array(state, dtype=np.int32, copy=True, order="C")
    acc = C.c_int64()
    lib().orc_metropolis(C.byref(sc), seed, step, int(sweeps), st.shape[0], _p(st), C.byref(acc))
    return st, acc.value


def metropolis_halfwidth(alpha, L):
    return lib().orc_metropolis_halfwidth(alpha, L)


def full_klist(s: System, nmax3):
    sc = s.c()
    nm = np.ascontiguousarray(nmax3, dtype=np.int32)
    K = lib().orc_full_klist(C.byref(sc), _p(nm), None, None)
    k = np.zeros((K, 3), dtype=np.int32)
    w = np.zeros(K)
    lib().orc_full_klist(C.byref(sc), _p(nm), _p(k), _p(w))
    return k, w


def image_coeff(s: System, l: int):
    sc = s.c()
    v = [C.c_double() for _ in range(6)]
    lib().orc_image_coeff(C.byref(sc), l, *[C.byref(x) for x in v])
    return tuple(x.value for x in v)  # gp, gm, dgp/dt, dgp/db, dgm/dt, dgm/db


def image_z(s: System, l: int, z: float):
    sc = s.c()
    zp, zm = C.c_double(), C.c_double()
    lib().orc_image_z(C.byref(sc), l, z, C.byref(zp), C.byref(zm))
    return zp.value, zm.value


def cM(s: System) -> float:
    sc = s.c()
    return lib().orc_cM(C.byref(sc))


def Y(s: System, kz: float):
    sc = s.c()
    yo = np.zeros(2); ye = np.zeros(2)
    lib().orc_Y(C.byref(sc), kz, _p(yo), _p(ye))
    return complex(yo[0], yo[1]), complex(ye[0], ye[1])


def sf_explicit(s: System, pos, q, kidx):
    sc = s.c()
    pos, q = _f64(pos), _f64(q)
    k = np.ascontiguousarray(kidx, dtype=np.int32)
    K = k.shape[0]
    out = [np.zeros(K, dtype=np.complex128) for _ in range(4)]
    lib().orc_sf_explicit(C.byref(sc), q.shape[0], _p(pos), _p(q), K, _p(k), *[_p(o) for o in out])
    return tuple(out)  # rho, rhobarM, drhobarM/dgt, drhobarM/dgb


def sf_recal(s: System, pos, q, kidx):
    sc = s.c()
    pos, q = _f64(pos), _f64(q)
    k = np.ascontiguousarray(kidx, dtype=np.int32)
    K = k.shape[0]
    out = [np.zeros(K, dtype=np.complex128) for _ in range(3)]
    lib().orc_sf_recal(C.byref(sc), q.shape[0], _p(pos), _p(q), K, _p(k), *[_p(o) for o in out])
    return tuple(out)  # rho, sigma, rhobarM


def rho_sigma(s: System, pos, q, kidx):
    sc = s.c()
    pos, q = _f64(pos), _f64(q)
    k = np.ascontiguousarray(kidx, dtype=np.int32)
    out = np.zeros((k.shape[0], 4))
    lib().orc_rho_sigma(C.byref(sc), q.shape[0], _p(pos), _p(q), k.shape[0], _p(k), _p(out))
    return out


def kspace(s: System, pos, q, kidx, W, mode=0, targets=None, want_force=True, want_dq=False,
           want_dgamma=False):
    """Energy terms {U_k, U_self, U_IBC}, forces, dU/dq and dU/dgamma for weights W."""
    sc = s.c()
    pos, q = _f64(pos), _f64(q)
    k = np.ascontiguousarray(kidx, dtype=np.int32)
    W = _f64(np.broadcast_to(np.asarray(W, dtype=np.float64), (k.shape[0],)))
    N = q.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = N if t is None else t.shape[0]
    energy = np.zeros(3)
    force = np.zeros((nt, 3)) if want_force else None
    dq = np.zeros(nt) if want_dq else None
    dg = np.zeros(2) if want_dgamma else None
    st = lib().orc_kspace(C.byref(sc), N, _p(pos), _p(q), k.shape[0], _p(k), _p(W), int(mode),
                          nt, _p(t), _p(energy), _p(force), _p(dq), _p(dg))
    if st != 0:
        raise MemoryError("oracle k-space allocation failed")
    return {"energy": energy, "force": force, "dUdq": dq, "dUdgamma": dg}


def rbe(s: System, pos, q, kidx, mode=0, **kw):
    """Random-batch estimator: weights S/P for the given batch of P wave vectors."""
    P = np.asarray(kidx).shape[0]
    return kspace(s, pos, q, kidx, S(s) / P, mode=mode, **kw)


def real_space(s: System, r_c, pos, q, targets=None):
    sc = s.c()
    pos, q = _f64(pos), _f64(q)
    N = q.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = N if t is None else t.shape[0]
    force = np.zeros((nt, 3))
    e = C.c_double()
    lib().orc_real_space(C.byref(sc), r_c, N, _p(pos), _p(q), nt, _p(t), _p(force), C.byref(e))
    return force, e.value


def auto_M(Lx, Ly, H, gt, gb, eps):
    return lib().orc_auto_M(Lx, Ly, H, gt, gb, eps)


def auto_Lz(Lx, Ly, H, M, alpha, eps):
    return lib().orc_auto_Lz(Lx, Ly, H, M, alpha, eps)


def auto_alpha(N, Lx, Ly, H):
    return lib().orc_auto_alpha(N, Lx, Ly, H)
