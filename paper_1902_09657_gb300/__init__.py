"""GB300 (sm_103a) k-space-preconditioned PDHG for non-Cartesian multi-coil MRI.

Ong, Uecker & Lustig, "Accelerating Non-Cartesian MRI Reconstruction Convergence using
k-space Preconditioning" (arXiv 1902.09657).  The compute path is the CUDA library
libkpdhg.so (C ABI in include/kpdhg.h); ``api.Plan`` is its Python binding.
"""
from ._build import build  # noqa: F401


def Plan(*args, **kwargs):
    """Create an :class:`api.Plan` (imports torch lazily)."""
    from .api import Plan as _Plan
    return _Plan(*args, **kwargs)
