"""Multi-threaded CSR products for timing the oracle on all host cores.

Test infrastructure only.  `CsrMv(A)` wraps a scipy CSR matrix (FP64 or
complex128) as a callable x -> A x computed by the oracle's own C kernel
(csrc/spmv_omp.c: one OpenMP thread per block of rows, entries of a row
summed in stored order).  `build()` compiles the kernel with gcc; where it
cannot be built, `CsrMv` falls back to scipy's single-threaded product and
`threads()` reports 1.
"""
import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "spmv_omp.c")
LIB = os.path.join(HERE, "_build", "liboracle_spmv.so")
_lib = None


def build():
    """Compile the OpenMP kernel (gcc -O2 -fopenmp); returns the library path."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    r = subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle spmv build failed:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        try:
            lib = ctypes.CDLL(build())
        except (OSError, RuntimeError):
            _lib = False
            return _lib
        p = ctypes.c_void_p
        for name in ("oracle_csr_mv_f64", "oracle_csr_mv_c128"):
            getattr(lib, name).argtypes = [ctypes.c_int64, p, p, p, p, p]
            getattr(lib, name).restype = None
        lib.oracle_spmv_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads():
    """OpenMP threads the kernel uses (1 if it is not available)."""
    lib = _load()
    return int(lib.oracle_spmv_threads()) if lib else 1


class CsrMv:
    """x -> A x for a square scipy sparse matrix A, FP64 or complex128."""

    def __init__(self, A):
        A = sp.csr_matrix(A)
        self.A = A
        self.n = A.shape[0]
        self.cplx = np.iscomplexobj(A.data)
        self.rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.col = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.val = np.ascontiguousarray(A.data, dtype=np.complex128 if self.cplx else np.float64)
        self.shape = A.shape

    def __call__(self, x):
        lib = _load()
        cplx = self.cplx or np.iscomplexobj(x)
        if not lib:
            return self.A.dot(x)
        dt = np.complex128 if cplx else np.float64
        x = np.ascontiguousarray(x, dtype=dt)
        if self.val.dtype == dt:
            val = self.val
        else:  # real A applied to a complex x: complex copy of the values, made once
            if getattr(self, "_valc", None) is None:
                self._valc = self.val.astype(dt)
            val = self._valc
        y = np.empty(self.n, dtype=dt)
        fn = lib.oracle_csr_mv_c128 if cplx else lib.oracle_csr_mv_f64
        fn(self.n, self.rowptr.ctypes.data, self.col.ctypes.data, val.ctypes.data, x.ctypes.data,
           y.ctypes.data)
        return y

    dot = __call__
