"""ctypes binding of include/pp.h: argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
vectors may be given as torch CUDA tensors (their data_ptr() is passed) or as
raw integer addresses; host vectors as numpy arrays.  A non-zero status raises
PPError (except PP_ERR_NOT_CONVERGED from pp_apply / pp_apply_host, which is
returned in the stats so the caller can inspect the last iterate).
"""
import ctypes
import os

import numpy as np

PP_OK = 0
PP_ERR_INVALID_ARG = -1
PP_ERR_NOT_CONVERGED = -2
PP_ERR_NONPRIMARY = -3
PP_ERR_SINGULAR = -4
PP_ERR_OOM = -5
PP_ERR_CUDA = -6
PP_ERR_TIMEOUT = -7
PP_ERR_STATE = -8
PP_ERR_UNSUPPORTED = -9

PP_F64, PP_F32, PP_C64, PP_C128 = 0, 1, 2, 3
PP_INVSQRT, PP_SQRT, PP_SIGN = -1, 1, 2
PP_CHEBYSHEV, PP_RITZ_LEJA, PP_HARMONIC_RITZ, PP_LSQ_CONTOUR, PP_NODES = 0, 1, 2, 3, 4
PP_LAPLACE2D5, PP_LAPLACE3D7, PP_CONVDIFF3D7_UPWIND, PP_WILSON4D_DHD, PP_WILSON4D_Q2 = 0, 1, 2, 3, 4
PP_LEFT, PP_RIGHT = 0, 1
PP_PREC_F64, PP_PREC_DW, PP_PREC_MIXED = 0, 1, 2
PP_ORTH_AUTO, PP_ORTH_LANCZOS, PP_ORTH_CGS2, PP_ORTH_DCGS2 = 0, 1, 2, 3

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libppsqrt.so")


class pp_opts(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("precision", ctypes.c_int32), ("orth", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("two_pass", ctypes.c_int32), ("clenshaw", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class pp_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("checks", ctypes.c_int32),
                ("breakdown", ctypes.c_int32), ("mvms", ctypes.c_int64),
                ("inner_products", ctypes.c_int64), ("est_err", ctypes.c_double),
                ("beta0", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("launches", ctypes.c_int64), ("chain_launches", ctypes.c_int64),
                ("chain_bytes", ctypes.c_double), ("chain_ms", ctypes.c_double),
                ("switch_iter", ctypes.c_int32), ("reserved_i", ctypes.c_int32),
                ("orth_ms", ctypes.c_double), ("small_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class PPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{pp_strerror(status)}: {msg}")
        self.status = status


_h = ctypes.c_void_p
_p = ctypes.c_void_p
SYMBOLS = {
    "pp_default_opts": (None, [ctypes.POINTER(pp_opts)]),
    "pp_create_csr": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int64, _p, _p, _p, ctypes.c_int32,
                                     ctypes.c_int32, _p]),
    "pp_create_stencil": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double), _p, ctypes.c_int32, _p]),
    "pp_set_opts": (ctypes.c_int, [_h, ctypes.POINTER(pp_opts)]),
    "pp_build_poly": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "pp_get_poly": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
    "pp_get_poly_nodes": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "pp_set_poly_nodes": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "pp_set_poly_lsq": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "pp_get_quadrature": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "pp_apply": (ctypes.c_int, [_h, ctypes.c_int32, _p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                _p, ctypes.POINTER(pp_stats)]),
    "pp_apply_host": (ctypes.c_int, [_h, ctypes.c_int32, _p, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_double, _p, ctypes.POINTER(pp_stats)]),
    "pp_apply_batch": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(_p), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_p),
                                      ctypes.c_int32, ctypes.c_double, _p, ctypes.POINTER(pp_stats)]),
    "pp_batch_create": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.POINTER(_h), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.c_int32, _p]),
    "pp_batch_apply": (ctypes.c_int, [_h, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.c_double,
                                      ctypes.POINTER(pp_stats)]),
    "pp_batch_destroy": (None, [_h]),
    "pp_autotune": (ctypes.c_int, [_h, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "pp_op_apply": (ctypes.c_int, [_h, _p, _p]),
    "pp_poly_apply": (ctypes.c_int, [_h, _p, _p]),
    "pp_poly_apply_static": (ctypes.c_int, [_h, _p, _p]),
    "pp_destroy": (None, [_h]),
    "pp_strerror": (ctypes.c_char_p, [ctypes.c_int32]),
    "pp_last_error": (ctypes.c_char_p, []),
    "pp_version": (ctypes.c_int32, []),
}

_LIB = None


def lib():
    """Load libppsqrt.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: build it with "
                               "paper_2401_06684_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SYMBOLS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc):
    if rc != PP_OK:
        raise PPError(rc, lib().pp_last_error().decode())


def pp_strerror(status):
    return lib().pp_strerror(status).decode()


def pp_last_error():
    return lib().pp_last_error().decode()


def pp_version():
    return lib().pp_version()


def pp_default_opts():
    o = pp_opts()
    lib().pp_default_opts(ctypes.byref(o))
    return o


def pp_create_csr(n, rowptr, col, val, dtype=PP_F64, is_hermitian=False, stream=None):
    h = _h()
    _check(lib().pp_create_csr(ctypes.byref(h), n, _ptr(rowptr), _ptr(col), _ptr(val), dtype,
                               1 if is_hermitian else 0, _stream(stream)))
    return h


def pp_create_stencil(kind, dims, params=None, links=None, dtype=PP_F64, stream=None):
    d = (ctypes.c_int64 * 4)(*(list(dims) + [0] * (4 - len(dims))))
    p = (ctypes.c_double * max(1, len(params or [])))(*(params or [0.0]))
    h = _h()
    _check(lib().pp_create_stencil(ctypes.byref(h), kind, d, p if params else None, _ptr(links), dtype,
                                   _stream(stream)))
    return h


def pp_set_opts(h, opts):
    _check(lib().pp_set_opts(h, ctypes.byref(opts)))


def pp_build_poly(h, degree, kind=PP_CHEBYSHEV, interval_ab=None):
    ab = (ctypes.c_double * 2)(*interval_ab) if interval_ab is not None else None
    _check(lib().pp_build_poly(h, degree, kind, ab))


def pp_get_poly(h):
    n = ctypes.c_int32()
    _check(lib().pp_get_poly(h, None, 0, ctypes.byref(n), None, None))
    c = (ctypes.c_double * n.value)()
    ab = (ctypes.c_double * 2)()
    img = (ctypes.c_double * 2)()
    _check(lib().pp_get_poly(h, c, n.value, ctypes.byref(n), ab, img))
    return np.array(c[:]), (ab[0], ab[1]), (img[0], img[1])


def pp_get_poly_nodes(h):
    """(kind, nodes, cap): the pp_poly_kind of q, its interpolation nodes in
    Leja order (complex array if any is complex) and the step scaling cap."""
    n = ctypes.c_int32()
    k = ctypes.c_int32()
    cap = ctypes.c_double()
    _check(lib().pp_get_poly_nodes(h, ctypes.byref(k), None, None, 0, ctypes.byref(n), None))
    xr = (ctypes.c_double * n.value)()
    xi = (ctypes.c_double * n.value)()
    _check(lib().pp_get_poly_nodes(h, ctypes.byref(k), xr, xi, n.value, ctypes.byref(n), ctypes.byref(cap)))
    re, im = np.array(xr[:]), np.array(xi[:])
    return k.value, (re + 1j * im if np.any(im != 0) else re), cap.value


def pp_set_poly_nodes(h, nodes, interval_ab=None):
    z = np.asarray(nodes)
    re = np.ascontiguousarray(np.real(z), dtype=np.float64)
    im = np.ascontiguousarray(np.imag(z), dtype=np.float64) if np.iscomplexobj(z) else None
    n = len(re)
    ab = (ctypes.c_double * 2)(*interval_ab) if interval_ab is not None else None
    _check(lib().pp_set_poly_nodes(h, re.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   im.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if im is not None else None,
                                   n, ab))


def pp_set_poly_lsq(h, degree, points):
    z = np.asarray(points)
    re = np.ascontiguousarray(np.real(z), dtype=np.float64)
    im = np.ascontiguousarray(np.imag(z), dtype=np.float64) if np.iscomplexobj(z) else None
    _check(lib().pp_set_poly_lsq(h, degree, re.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 im.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if im is not None else None,
                                 len(re)))


def pp_get_quadrature(h):
    K = ctypes.c_int32()
    _check(lib().pp_get_quadrature(h, None, None, 0, ctypes.byref(K)))
    s = (ctypes.c_double * K.value)()
    w = (ctypes.c_double * K.value)()
    _check(lib().pp_get_quadrature(h, s, w, K.value, ctypes.byref(K)))
    return np.array(s[:]), np.array(w[:])


def pp_apply(h, f, b, x, m_max=200, tol=1e-10, nrhs=1):
    st = pp_stats()
    rc = lib().pp_apply(h, f, _ptr(b), nrhs, m_max, tol, _ptr(x), ctypes.byref(st))
    if rc not in (PP_OK, PP_ERR_NOT_CONVERGED):
        _check(rc)
    st.status = rc
    return st


def pp_apply_host(h, f, b, x, m_max=200, tol=1e-10, nrhs=1):
    st = pp_stats()
    rc = lib().pp_apply_host(h, f, _ptr(b), nrhs, m_max, tol, _ptr(x), ctypes.byref(st))
    if rc not in (PP_OK, PP_ERR_NOT_CONVERGED):
        _check(rc)
    st.status = rc
    return st


def pp_apply_batch(handles, fs, bs, xs, nrhs=None, m_max=200, tol=1e-10, stream=None):
    """Batched solves; returns one pp_stats per handle (see pp.h)."""
    n = len(handles)
    nrhs = nrhs or [1] * n
    hs = (_h * n)(*[h.value if hasattr(h, "value") else h for h in handles])
    fa = (ctypes.c_int32 * n)(*fs)
    ba = (_p * n)(*[_ptr(b) for b in bs])
    xa = (_p * n)(*[_ptr(x) for x in xs])
    ra = (ctypes.c_int64 * n)(*nrhs)
    st = (pp_stats * n)()
    rc = lib().pp_apply_batch(hs, n, fa, ba, ra, xa, m_max, tol, _stream(stream), st)
    if rc not in (PP_OK, PP_ERR_NOT_CONVERGED):
        _check(rc)
    return list(st)


def pp_batch_create(handles, fs, nrhs=None, m_max=200, stream=None):
    """A batch plan for the processes of pp_apply_batch (see pp.h); returns its handle."""
    n = len(handles)
    nrhs = nrhs or [1] * n
    hs = (_h * n)(*[h.value if hasattr(h, "value") else h for h in handles])
    fa = (ctypes.c_int32 * n)(*fs)
    ra = (ctypes.c_int64 * n)(*nrhs)
    b = _h()
    _check(lib().pp_batch_create(ctypes.byref(b), hs, n, fa, ra, m_max, _stream(stream)))
    b.n_handles = n
    return b


def pp_batch_apply(b, bs, xs, tol=1e-10):
    """Solve the plan's processes for the right-hand sides bs into xs; one pp_stats per handle."""
    n = len(bs)
    ba = (_p * n)(*[_ptr(v) for v in bs])
    xa = (_p * n)(*[_ptr(v) for v in xs])
    st = (pp_stats * n)()
    rc = lib().pp_batch_apply(b, ba, xa, tol, st)
    if rc not in (PP_OK, PP_ERR_NOT_CONVERGED):
        _check(rc)
    return list(st)


def pp_batch_destroy(b):
    lib().pp_batch_destroy(b)


def pp_autotune(h, tol, max_degree=64):
    d = ctypes.c_int32()
    _check(lib().pp_autotune(h, tol, max_degree, ctypes.byref(d)))
    return d.value


def pp_op_apply(h, x, y):
    _check(lib().pp_op_apply(h, _ptr(x), _ptr(y)))


def pp_poly_apply(h, x, y):
    _check(lib().pp_poly_apply(h, _ptr(x), _ptr(y)))


def pp_poly_apply_static(h, x, y):
    _check(lib().pp_poly_apply_static(h, _ptr(x), _ptr(y)))


PP_STATIC_MAX_N = 262144


def pp_destroy(h):
    if h is not None:
        lib().pp_destroy(h)
