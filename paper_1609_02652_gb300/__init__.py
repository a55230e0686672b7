"""GB300 (sm_103a) library for the data-parallel hot path of polynomial-filtered
mass-preconditioned HMC.  The compute lives in ``libpfmp.so`` (hand-written CUDA behind
the C-ABI of ``include/pfmp.h``); ``capi`` is its ctypes binding and ``fields`` a few
helpers that allocate device buffers with PyTorch.  There is no CPU fallback: the
binding raises if the library is not built.
"""
from . import capi  # noqa: F401

__all__ = ["capi"]
