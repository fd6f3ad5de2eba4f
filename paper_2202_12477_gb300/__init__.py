"""GB300-native matrix-free spectral-element screened-Poisson operator and CG.

The compute path is the CUDA library built from ``csrc/`` (``build.build()``),
reached through the C ABI in ``include/hipbone_gb300.h``; ``hb`` is its ctypes
binding.
"""
__all__ = ["hb", "build", "inputs", "accounting"]
