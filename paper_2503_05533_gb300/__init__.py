"""libmlmc: the MPML hot path (arXiv 2503.05533) as hand-written CUDA for GB300 (sm_103a).

The compute lives in ``libmlmc.so`` (C ABI, include/libmlmc.h); ``capi``
is the thin ctypes binding with the same function names and ``autograd``
wraps the adjoint gradient as a ``torch.autograd.Function``.
"""
from . import capi  # noqa: F401
from .capi import *  # noqa: F401,F403

__all__ = [n for n in dir(capi) if n.startswith(("mlmc_", "MLMC_", "make_problem", "MlmcError", "result_dict"))]
