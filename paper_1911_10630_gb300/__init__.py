"""GB300-native pair-Poisson exact exchange (arXiv:1911.10630 hot path).

The CUDA library sits behind a C ABI (``include/exx.h``); ``exx`` is its thin
ctypes binding. Importing the package loads nothing; the binding loads the
shared library on first use and raises if it is missing.
"""
__all__ = ["synth", "exx"]
