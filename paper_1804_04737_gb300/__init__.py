"""GB300-native dense tableau simplex (arXiv:1804.04737, Sec. 2-3).

The compute runs in the CUDA library ``_lib/libgbsimplex.so`` (C ABI in
``include/gbsimplex.h``); :mod:`.capi` is its ctypes binding and
:mod:`.lpgen` the seeded synthetic-LP generators.
"""
from . import lpgen  # noqa: F401

__all__ = ["capi", "lpgen", "build"]
