"""GB300 (sm_103a) implementation of the FED-FEM hot path (Zhang & Chauhan, arXiv:1909.03355).

The compute path is libfedfem.so (CUDA, C ABI in include/fedfem.h); this package is its thin
Python binding.  Import is light: the library is loaded on first use and its absence raises.
"""
from .capi import FedFemError, library_path, load  # noqa: F401


def FedFem(*args, **kw):
    from .fedfem import FedFem as _F
    return _F(*args, **kw)
