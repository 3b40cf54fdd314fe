"""GB300-native batched Monte Carlo graph propagation (SIR, SIS, IC, LT).

The compute path is libfsgp.so (hand-written CUDA for sm_103a, C ABI in
include/fsgp.h); ``fsgp`` is its thin ctypes binding.
"""
from . import fsgp  # noqa: F401

__all__ = ["fsgp"]
