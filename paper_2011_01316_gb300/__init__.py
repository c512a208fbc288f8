"""GB300-native exponential-DG hot path (arXiv 2011.01316, Kang & Bui-Thanh).

The compute path lives in the CUDA library ``libexpdg.so`` built from
``csrc/`` (C-ABI declared in ``include/expdg.h``).  ``expdg`` is the thin
ctypes binding with the same names; ``inputs`` generates seeded synthetic
states.  Importing this package does not load the library; the binding
loads it on first use and raises if it is missing.
"""

__all__ = ["inputs", "expdg"]
