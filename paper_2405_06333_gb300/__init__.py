"""GB300 (sm_103a) random-batch Ewald k-space force for dielectrically confined
quasi-2D Coulomb systems (RBE2D, arXiv 2405.06333).

- ``binding``: ctypes binding of the C ABI in include/rbe2d.h (librbe2d.so).
- ``rbe2d``: torch-tensor wrapper (``RBE2D``) and ``RBE2DEnergy`` autograd.Function.
- ``synthetic``: seeded synthetic inputs.
- ``build``: compiles librbe2d.so for sm_103a.
Importing the package does not load CUDA; the library is loaded on first use.
"""

__all__ = ["binding", "synthetic", "build"]


def __getattr__(name):
    if name in ("RBE2D", "RBE2DEnergy"):
        from . import rbe2d as _m
        return getattr(_m, name)
    raise AttributeError(name)
