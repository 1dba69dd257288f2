"""GB300-native polynomially preconditioned Krylov library for A^{-1/2} b and A^{1/2} b.

The compute path is the C-ABI shared library built from ``csrc/`` (see
``include/pp.h``); ``pp`` is a thin ctypes binding with the same entry-point
names.  Importing the package does not load the library: ``pp.lib()`` does,
and raises if it has not been built.
"""
from . import pp  # noqa: F401
