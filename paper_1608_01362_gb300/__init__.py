"""GB300-native segmented pull gather (Cagra: CSR segmenting + frequency-based
clustering, arXiv 1608.01362).

The compute lives in the CUDA library libcagra_gb.so (C ABI in
include/cagra_gb.h); `cagra` is its thin ctypes binding and `pipeline` chains
the calls a user makes (degrees -> clustering -> segmenting -> iterations).
"""
from . import cagra  # noqa: F401

__all__ = ["cagra"]
