"""Thin ctypes binding of librbe2d (include/rbe2d.h): argument marshalling only.

Every function keeps the C name and takes torch tensors (device pointers) or, with
RBE2D_HOST_BUFFERS, numpy arrays / CPU tensors (host pointers).  All arithmetic runs in
the CUDA kernels of librbe2d.so; there is no CPU path.  Loading fails loudly if the
library has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbe2d.so")

RBE2D_OK = 0
RBE2D_EINVAL = -1
RBE2D_ENONNEUTRAL = -2
RBE2D_ERANGE = -3
RBE2D_ECUDA = -4
RBE2D_ETIMEOUT = -5
RBE2D_ESAMPLER = -6
RBE2D_ENOMEM = -7

RBE2D_FP64 = 0
RBE2D_FP32_MIXED = 1

RBE2D_KSPACE = 1
RBE2D_REAL = 2
RBE2D_IBC = 4
RBE2D_ENERGY = 8
RBE2D_POTENTIAL = 16
RBE2D_HOST_BUFFERS = 32
RBE2D_VALIDATE = 64
RBE2D_INPUT_F32 = 128
RBE2D_REUSE_SF = 256
RBE2D_ACCUMULATE = 512

_STATUS_NAMES = {0: "RBE2D_OK", -1: "RBE2D_EINVAL", -2: "RBE2D_ENONNEUTRAL", -3: "RBE2D_ERANGE",
                 -4: "RBE2D_ECUDA", -5: "RBE2D_ETIMEOUT", -6: "RBE2D_ESAMPLER", -7: "RBE2D_ENOMEM"}


class rbe2d_params(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("H", C.c_double), ("Lz", C.c_double),
                ("gamma_top", C.c_double), ("gamma_bot", C.c_double), ("M", C.c_int),
                ("alpha", C.c_double), ("r_c", C.c_double), ("P", C.c_int), ("seed", C.c_uint64),
                ("eps", C.c_double), ("precision", C.c_int), ("coulomb_k", C.c_double),
                ("real_space", C.c_int), ("skin", C.c_double)]


class rbe2d_md_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gamma", C.c_double), ("kT", C.c_double), ("mass", C.c_double),
                ("sigma_lj", C.c_double), ("eps_lj", C.c_double), ("sigma_wall", C.c_double),
                ("eps_wall", C.c_double), ("noise_seed", C.c_uint64), ("force_flags", C.c_int)]


RBE2D_MD_FORCE = 1
RBE2D_MD_STEP = 2

# kernel classes of the per-kernel timer (rbe2d_timer_enable / rbe2d_timer_read)
TIMER_NAMES = ("sample", "pack", "structure_factor", "fold", "force", "real_space", "md")
RBE2D_TIMER_COUNT = len(TIMER_NAMES)
RBE2D_TIMER_ALL = (1 << RBE2D_TIMER_COUNT) - 1


class RBE2DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded librbe2d.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"librbe2d.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, u64, d, i = C.c_void_p, C.c_int64, C.c_uint64, C.c_double, C.c_int
        L.rbe2d_init.argtypes = [C.POINTER(rbe2d_params), i64, vp, C.POINTER(vp)]
        L.rbe2d_destroy.argtypes = [vp]
        L.rbe2d_last_error.argtypes = [vp]
        L.rbe2d_last_error.restype = C.c_char_p
        L.rbe2d_get_derived.argtypes = [vp, vp, vp, vp, vp, vp]
        L.rbe2d_sample_k.argtypes = [vp, u64, vp]
        L.rbe2d_set_k.argtypes = [vp, vp]
        L.rbe2d_structure_factor.argtypes = [vp, i64, vp, vp, i, vp]
        L.rbe2d_force.argtypes = [vp, i64, vp, vp, i, vp, vp, vp]
        L.rbe2d_energy_backward.argtypes = [vp, i64, vp, vp, i, d, vp, vp, vp]
        L.rbe2d_sync_status.argtypes = [vp]
        L.rbe2d_autotune.argtypes = [vp, i64, vp, vp, i, vp, vp]
        L.rbe2d_autotune.restype = C.c_int
        L.rbe2d_set_tuning.argtypes = [vp, vp]
        L.rbe2d_set_tuning.restype = C.c_int
        L.rbe2d_autotune_potential.argtypes = [vp, i64, vp, vp, i, vp, vp, vp]
        L.rbe2d_autotune_potential.restype = C.c_int
        L.rbe2d_set_tuning_potential.argtypes = [vp, vp]
        L.rbe2d_set_tuning_potential.restype = C.c_int
        L.rbe2d_charge_sums.argtypes = [vp, vp]
        L.rbe2d_charge_sums.restype = C.c_int
        L.rbe2d_set_structure_factor.argtypes = [vp, i64, vp, vp]
        L.rbe2d_set_structure_factor.restype = C.c_int
        L.rbe2d_sample_k_dev.argtypes = [vp, vp, vp]
        L.rbe2d_sample_k_dev.restype = C.c_int
        L.rbe2d_md_step.argtypes = [vp, i64, vp, vp, vp, vp, vp, C.POINTER(rbe2d_md_params), i, vp]
        L.rbe2d_md_step.restype = C.c_int
        L.rbe2d_md_list_stats.argtypes = [vp, vp, vp]
        L.rbe2d_md_list_stats.restype = C.c_int
        L.rbe2d_batch_init.argtypes = [C.POINTER(rbe2d_params), i, vp, vp, C.POINTER(vp)]
        L.rbe2d_batch_destroy.argtypes = [vp]
        L.rbe2d_batch_last_error.argtypes = [vp]
        L.rbe2d_batch_last_error.restype = C.c_char_p
        L.rbe2d_batch_force.argtypes = [vp, u64, vp, vp, i, vp, vp]
        L.rbe2d_batch_sync_status.argtypes = [vp]
        L.rbe2d_batch_autotune.argtypes = [vp, vp, vp, vp, vp]
        L.rbe2d_batch_set_wait.argtypes = [vp, d, i]
        L.rbe2d_batch_set_tuning.argtypes = [vp, vp]
        for name in ("rbe2d_batch_init", "rbe2d_batch_destroy", "rbe2d_batch_force", "rbe2d_batch_sync_status",
                     "rbe2d_batch_autotune", "rbe2d_batch_set_wait", "rbe2d_batch_set_tuning"):
            getattr(L, name).restype = C.c_int
        L.rbe2d_metropolis_reset.argtypes = [vp, vp]
        L.rbe2d_metropolis_reset.restype = C.c_int
        L.rbe2d_sample_k_metropolis.argtypes = [vp, u64, i, vp]
        L.rbe2d_sample_k_metropolis.restype = C.c_int
        L.rbe2d_metropolis_accepted.argtypes = [vp, vp]
        L.rbe2d_metropolis_accepted.restype = C.c_int
        L.rbe2d_force_lattice.argtypes = [vp, i64, vp, vp, i, vp, vp, vp, vp]
        L.rbe2d_force_lattice.restype = C.c_int
        L.rbe2d_kernel_launches.argtypes = [vp]
        L.rbe2d_kernel_launches.restype = C.c_int
        L.rbe2d_timer_enable.argtypes = [vp, i, C.c_uint]
        L.rbe2d_timer_enable.restype = C.c_int
        L.rbe2d_timer_read.argtypes = [vp, vp, vp]
        L.rbe2d_timer_read.restype = C.c_int
        L.rbe2d_pipe_probe.argtypes = [vp]
        L.rbe2d_pipe_probe.restype = C.c_int
        L.rbe2d_structure_factor_noalloc.argtypes = [d, d, d, i64, vp, vp, i, vp, vp, vp]
        L.rbe2d_structure_factor_noalloc.restype = C.c_int
        for name in ("rbe2d_init", "rbe2d_destroy", "rbe2d_get_derived", "rbe2d_sample_k", "rbe2d_set_k",
                     "rbe2d_structure_factor", "rbe2d_force", "rbe2d_energy_backward", "rbe2d_sync_status"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(ctx, code):
    if code != RBE2D_OK:
        msg = lib().rbe2d_last_error(ctx).decode(errors="replace")
        raise RBE2DError(code, msg)


def rbe2d_init(params: rbe2d_params, n_max: int, stream=None):
    """Create a context; stream is a torch.cuda.Stream, a raw handle or None (current stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    ctx = C.c_void_p()
    code = lib().rbe2d_init(C.byref(params), int(n_max), C.c_void_p(h), C.byref(ctx))
    if code != RBE2D_OK:
        raise RBE2DError(code, lib().rbe2d_last_error(None).decode(errors="replace"))
    return ctx


def rbe2d_destroy(ctx):
    return lib().rbe2d_destroy(ctx)


def rbe2d_last_error(ctx):
    return lib().rbe2d_last_error(ctx).decode(errors="replace")


def rbe2d_get_derived(ctx):
    S, Lz, a, rc = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    M = C.c_int()
    _check(ctx, lib().rbe2d_get_derived(ctx, C.byref(S), C.byref(Lz), C.byref(M), C.byref(a), C.byref(rc)))
    return {"S": S.value, "Lz": Lz.value, "M": M.value, "alpha": a.value, "r_c": rc.value}


def rbe2d_sample_k(ctx, step: int, k_idx_out=None):
    _check(ctx, lib().rbe2d_sample_k(ctx, int(step), _ptr(k_idx_out)))


def rbe2d_set_k(ctx, k_idx):
    _check(ctx, lib().rbe2d_set_k(ctx, _ptr(k_idx)))


def rbe2d_structure_factor(ctx, N, pos, q, flags=0, rho_out=None):
    _check(ctx, lib().rbe2d_structure_factor(ctx, int(N), _ptr(pos), _ptr(q), int(flags), _ptr(rho_out)))


def rbe2d_force(ctx, N, pos, q, flags, force_out, phi_out=None, energy_out=None):
    _check(ctx, lib().rbe2d_force(ctx, int(N), _ptr(pos), _ptr(q), int(flags), _ptr(force_out), _ptr(phi_out),
                                  _ptr(energy_out)))


def rbe2d_energy_backward(ctx, N, pos, q, flags, grad_energy, dpos=None, dq=None, dgamma=None):
    _check(ctx, lib().rbe2d_energy_backward(ctx, int(N), _ptr(pos), _ptr(q), int(flags), float(grad_energy),
                                            _ptr(dpos), _ptr(dq), _ptr(dgamma)))


def rbe2d_sync_status(ctx):
    _check(ctx, lib().rbe2d_sync_status(ctx))


def rbe2d_autotune(ctx, N, pos, q, flags, force_scratch):
    import numpy as np
    choice = np.zeros(4, dtype=np.int32)
    _check(ctx, lib().rbe2d_autotune(ctx, int(N), _ptr(pos), _ptr(q), int(flags), _ptr(force_scratch),
                                     choice.ctypes.data))
    return {"sf_poly": int(choice[0]), "force_poly": int(choice[1]), "sf_shape": int(choice[2]),
            "force_shape": int(choice[3])}


def rbe2d_set_tuning(ctx, sf_poly, force_poly, sf_shape=0, force_shape=0):
    import numpy as np
    choice = np.array([sf_poly, force_poly, sf_shape, force_shape], dtype=np.int32)
    _check(ctx, lib().rbe2d_set_tuning(ctx, choice.ctypes.data))


def rbe2d_autotune_potential(ctx, N, pos, q, flags, force_scratch, phi_scratch):
    import numpy as np
    choice = np.zeros(2, dtype=np.int32)
    _check(ctx, lib().rbe2d_autotune_potential(ctx, int(N), _ptr(pos), _ptr(q), int(flags), _ptr(force_scratch),
                                               _ptr(phi_scratch), choice.ctypes.data))
    return {"potential_poly": int(choice[0]), "potential_shape": int(choice[1])}


def rbe2d_set_tuning_potential(ctx, poly, shape=0):
    import numpy as np
    choice = np.array([poly, shape], dtype=np.int32)
    _check(ctx, lib().rbe2d_set_tuning_potential(ctx, choice.ctypes.data))


def rbe2d_metropolis_reset(ctx, k_start=None):
    _check(ctx, lib().rbe2d_metropolis_reset(ctx, _ptr(k_start)))


def rbe2d_sample_k_metropolis(ctx, step, sweeps, k_idx_out=None):
    _check(ctx, lib().rbe2d_sample_k_metropolis(ctx, int(step), int(sweeps), _ptr(k_idx_out)))


def rbe2d_metropolis_accepted(ctx):
    v = C.c_uint64()
    _check(ctx, lib().rbe2d_metropolis_accepted(ctx, C.byref(v)))
    return v.value


def rbe2d_force_lattice(ctx, N, pos, q, flags, nmax, force_out, phi_out=None, energy_out=None):
    import numpy as np
    nm = np.ascontiguousarray(nmax, dtype=np.int32)
    assert nm.shape == (3,)
    _check(ctx, lib().rbe2d_force_lattice(ctx, int(N), _ptr(pos), _ptr(q), int(flags), nm.ctypes.data,
                                          _ptr(force_out), _ptr(phi_out), _ptr(energy_out)))


def rbe2d_kernel_launches():
    """Kernels this library has enqueued in this process so far."""
    v = C.c_uint64()
    st = lib().rbe2d_kernel_launches(C.byref(v))
    if st != RBE2D_OK:
        raise RBE2DError(st, "rbe2d_kernel_launches failed")
    return v.value


def rbe2d_pipe_probe():
    """{"mufu", "fp32_fma", "fp64_fma"}: measured results per clock per SM, and "sm_mhz"."""
    import numpy as np
    out = np.zeros(4, dtype=np.float64)
    st = lib().rbe2d_pipe_probe(out.ctypes.data)
    if st != RBE2D_OK:
        raise RBE2DError(st, "rbe2d_pipe_probe failed")
    return {"mufu": float(out[0]), "fp32_fma": float(out[1]), "fp64_fma": float(out[2]), "sm_mhz": float(out[3])}


def rbe2d_timer_enable(ctx, capacity, classes=TIMER_NAMES):
    """Time up to `capacity` launches of each named kernel class (0 disables)."""
    mask = 0
    for name in classes:
        mask |= 1 << TIMER_NAMES.index(name)
    _check(ctx, lib().rbe2d_timer_enable(ctx, int(capacity), mask if capacity else 0))


def rbe2d_timer_read(ctx):
    """{kernel class: (summed device ms, recorded launches)}; clears the records."""
    import numpy as np
    ms = np.zeros(RBE2D_TIMER_COUNT, dtype=np.float64)
    n = np.zeros(RBE2D_TIMER_COUNT, dtype=np.int64)
    _check(ctx, lib().rbe2d_timer_read(ctx, ms.ctypes.data, n.ctypes.data))
    return {name: (float(ms[k]), int(n[k])) for k, name in enumerate(TIMER_NAMES)}


def rbe2d_charge_sums(ctx, sums_out):
    _check(ctx, lib().rbe2d_charge_sums(ctx, _ptr(sums_out)))


def rbe2d_set_structure_factor(ctx, N, rho, sums):
    _check(ctx, lib().rbe2d_set_structure_factor(ctx, int(N), _ptr(rho), _ptr(sums)))


def rbe2d_sample_k_dev(ctx, step_dev, k_idx_out=None):
    _check(ctx, lib().rbe2d_sample_k_dev(ctx, _ptr(step_dev), _ptr(k_idx_out)))


def rbe2d_md_step(ctx, N, pos, vel, q, force_inout, step_dev, md: rbe2d_md_params, mode, stats_dev=None):
    _check(ctx, lib().rbe2d_md_step(ctx, int(N), _ptr(pos), _ptr(vel), _ptr(q), _ptr(force_inout), _ptr(step_dev),
                                    C.byref(md), int(mode), _ptr(stats_dev)))


def rbe2d_md_list_stats(ctx):
    """{"enabled": bool, "builds": int}: the MD pair lists of the context."""
    en, nb = C.c_int(), C.c_uint64()
    _check(ctx, lib().rbe2d_md_list_stats(ctx, C.byref(en), C.byref(nb)))
    return {"enabled": bool(en.value), "builds": int(nb.value)}


def rbe2d_structure_factor_noalloc(Lx, Ly, Lz, N, pos, q, P, k_idx, rho_out, stream=None):
    """Structure factors with no context and no device allocation (fixed 4 MiB scratch
    inside the library, P <= 512).  For callers that cannot allocate on their call path."""
    h = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    code = lib().rbe2d_structure_factor_noalloc(float(Lx), float(Ly), float(Lz), int(N), _ptr(pos), _ptr(q),
                                                int(P), _ptr(k_idx), _ptr(rho_out), C.c_void_p(h))
    if code != RBE2D_OK:
        raise RBE2DError(code, "rbe2d_structure_factor_noalloc: P must be in [1, 512], sizes and pointers valid")


def _bcheck(batch, code):
    if code != RBE2D_OK:
        raise RBE2DError(code, lib().rbe2d_batch_last_error(batch).decode(errors="replace"))


def rbe2d_batch_init(per_sys, offsets, stream=None):
    """per_sys: sequence of rbe2d_params; offsets: n_sys + 1 int64 (host)."""
    import numpy as np
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    arr = (rbe2d_params * len(per_sys))(*per_sys)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    b = C.c_void_p()
    code = lib().rbe2d_batch_init(arr, len(per_sys), off.ctypes.data, C.c_void_p(h), C.byref(b))
    if code != RBE2D_OK:
        raise RBE2DError(code, "rbe2d_batch_init: invalid per-system parameters or offsets")
    return b


def rbe2d_batch_destroy(batch):
    return lib().rbe2d_batch_destroy(batch)


def rbe2d_batch_last_error(batch):
    return lib().rbe2d_batch_last_error(batch).decode(errors="replace")


def rbe2d_batch_force(batch, step, pos, q, flags, force_out, energy_out=None):
    _bcheck(batch, lib().rbe2d_batch_force(batch, int(step), _ptr(pos), _ptr(q), int(flags), _ptr(force_out),
                                           _ptr(energy_out)))


def rbe2d_batch_sync_status(batch):
    _bcheck(batch, lib().rbe2d_batch_sync_status(batch))


def rbe2d_batch_set_wait(batch, seconds, withhold_sys=-1):
    """Bound of the force items' wait (s) and the system whose fold is kept unpublished
    (host-side fault injection for timeout tests; -1: none)."""
    _bcheck(batch, lib().rbe2d_batch_set_wait(batch, float(seconds), int(withhold_sys)))


def rbe2d_batch_set_tuning(batch, sf_chunk, f_chunk, grid, variant):
    import numpy as np
    choice = np.array([sf_chunk, f_chunk, grid, variant], dtype=np.int32)
    _bcheck(batch, lib().rbe2d_batch_set_tuning(batch, choice.ctypes.data))


def rbe2d_batch_autotune(batch, pos, q, force_out):
    import numpy as np
    choice = np.zeros(4, dtype=np.int32)
    _bcheck(batch, lib().rbe2d_batch_autotune(batch, _ptr(pos), _ptr(q), _ptr(force_out), choice.ctypes.data))
    return {"sf_chunk": int(choice[0]), "f_chunk": int(choice[1]), "grid": int(choice[2]), "variant": int(choice[3])}


def status_code(fn, *a, **kw):
    """Call a binding function and return its status code instead of raising."""
    try:
        fn(*a, **kw)
        return RBE2D_OK
    except RBE2DError as e:
        return e.code
