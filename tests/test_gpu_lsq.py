"""GPU parity of the least-squares contour polynomial (Sec. 5.3) through the
C ABI against the oracle (oracle/lsq.py).

The library evaluates q in Newton form at degree + 1 Leja points of the
contour; the oracle evaluates it through its orthonormal basis recurrence
(the evaluation Sec. 5.3 describes).  q(A) v: 1e-10 (FP64), 5e-10
(double-word), 2e-7 (deg + 1) (FP32) relative; solves 1e-10 against the
exact result (mixed: within max(3 x the double-word error, tol)).
"""
import functools

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import exact, krylov, lsq, operators as ops
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"f64": 0, "dw": 1, "mixed": 2}


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def cd_contour(dims, npts=600):
    # a thin contour symmetric about the real axis around the (real) spectrum
    # of the convection-diffusion operator, kept off |z| < a/2
    a, b = ops.convdiff_interval(dims, 0.5)
    th = np.array([a, b, 0.5 * (a + b) + 0.05 * (b - a) * 1j, 0.5 * (a + b) - 0.05 * (b - a) * 1j])
    return lsq.contour(th, 0.5 * a, npts)


def set_prec(pp, h, prec, side=0):
    o = pp.pp_default_opts()
    o.precision = PREC[prec]
    o.side = side
    pp.pp_set_opts(h, o)


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("degree", [0, 1, 4, 9, 16])
@pytest.mark.parametrize("csr", [False, True], ids=["stencil", "csr"])
def test_lsq_poly_apply(csr, degree, prec):
    pp = load()
    dims = (13, 11, 9) if not csr else (9, 8, 7)
    A = ops.convdiff(dims, 0.5)
    n = A.shape[0]
    keep = []
    if csr:
        rp, col, val = synth.stencil_csr("convdiff3d7", dims, 0.5)
        keep = [dev(rp), dev(col), dev(val)]
        h = pp.pp_create_csr(n, *keep, is_hermitian=False)
    else:
        h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        z = cd_contour(dims)
        pp.pp_set_poly_lsq(h, degree, z)
        set_prec(pp, h, prec)
        P, H = lsq.basis(z, degree + 1)
        al = lsq.coeffs(P, z ** -0.5)
        v = synth.rhs(n, 7)
        yd = torch.empty(n, dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(h, dev(v), yd)
        ref = lsq.apply(A.dot, H, al, len(z), v)
        tol = {"f64": 1e-10, "dw": 5e-10, "mixed": 2e-7 * (degree + 1)}[prec]
        assert rel(host(yd), ref) < tol
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
@pytest.mark.parametrize("degree", [4, 12])
def test_lsq_solve_convdiff(degree, side, f, prec):
    pp = load()
    dims = (13, 11, 9)
    A = ops.convdiff(dims, 0.5)
    n = A.shape[0]
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_set_poly_lsq(h, degree, cd_contour(dims))
        b = synth.rhs(n, 0)
        xs = exact.dense_fun(A.toarray(), b, 0.5 * f, hermitian=False)
        xd = torch.empty(n, dtype=torch.float64, device="cuda")
        if prec == "mixed":
            set_prec(pp, h, "dw", side)
            pp.pp_apply(h, f, dev(b), xd, m_max=400, tol=1e-12)
            err_dw = rel(host(xd), xs)
        set_prec(pp, h, prec, side)
        st = pp.pp_apply(h, f, dev(b), xd, m_max=400, tol=1e-12)
        assert st.status == pp.PP_OK
        err = rel(host(xd), xs)
        assert err < 1e-10 if prec != "mixed" else err <= max(3 * err_dw, 1e-12)
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("degree", [3, 8, 16])
def test_lsq_build_on_segment(degree, prec):
    # pp_build_poly(PP_LSQ_CONTOUR) with the closed-form spectrum of the 2D
    # Laplacian: the least-squares q on its segment, then a solve
    pp = load()
    dims = (61, 37)
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    try:
        set_prec(pp, h, prec)
        pp.pp_build_poly(h, degree, pp.PP_LSQ_CONTOUR)
        a, b = ops.laplace_interval(dims)
        seg = np.linspace(a, b, max(2000, 20 * (degree + 1)))
        P, H = lsq.basis(seg, degree + 1)
        al = lsq.coeffs(P, seg ** -0.5)
        A = ops.laplace(dims)
        v = synth.rhs(A.shape[0], 3)
        yd = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(h, dev(v), yd)
        assert rel(host(yd), lsq.apply(A.dot, H, al, len(seg), v)) < (1e-10 if prec == "f64" else 5e-10)
        bb = synth.rhs(A.shape[0], 0)
        xd = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, -1, dev(bb), xd, m_max=600, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), exact.separable_fun(dims, bb, -0.5)) < 1e-10
    finally:
        pp.pp_destroy(h)


@functools.lru_cache(maxsize=None)
def graph():
    src, dst = synth.directed_powerlaw_graph(1500, 12000, seed=5)
    return synth.graph_laplacian_csr(1500, src, dst)


@pytest.mark.parametrize("degree", [3, 7])
def test_lsq_build_from_ritz_values_graph(degree):
    # Example 3's right-hand side of Table 3: the contour from the Ritz values
    # of 60 Arnoldi steps; q must be positive on it, and L^{1/2} e_i must match
    # the oracle's plain Arnoldi reference where q is positive on the spectrum
    pp = load()
    rp, col, val = graph()
    N = 1500
    L = sp.csr_matrix((val, col, rp), shape=(N, N))
    keep = [dev(rp), dev(col), dev(val)]
    h = pp.pp_create_csr(N, *keep, is_hermitian=False)
    try:
        pp.pp_build_poly(h, degree, pp.PP_LSQ_CONTOUR)
        kind, x, _ = pp.pp_get_poly_nodes(h)
        a, _, img = pp.pp_get_poly(h)
        assert kind == pp.PP_LSQ_CONTOUR and img[0] > 0
        b = synth.unit_vector(N, 4)
        ref = krylov.pp_arnoldi(L.dot, b, 0.5, m_max=N, tol=1e-13, k_chk=8, orth="cgs2")["x"]
        xd = torch.empty(N, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, pp.PP_SQRT, dev(b), xd, m_max=800, tol=1e-11)
        assert st.status == pp.PP_OK
        assert rel(host(xd), ref) < 5e-8
    finally:
        pp.pp_destroy(h)


# ---- complex operator (Sec. 6, Example 2's Q^2 with mu != 0): complex q on a contour
# with no symmetry about the real axis

def _q2_handle(pp, dims):
    from tests.test_gpu_sign import Q2
    return Q2(pp, dims, synth.wilson_links(dims, 1))


def _skew_ellipse(npts=500):
    # an ellipse in the right half-plane, tilted off the real axis (centre 5 + 0.6i,
    # semi-axes 4 and 1.2): Re z in [1, 9], not symmetric about the real axis
    t = 2.0 * np.pi * np.arange(npts) / npts
    return (5.0 + 0.6j) + 4.0 * np.cos(t) + 1.2j * np.sin(t)


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("degree", [1, 4, 9])
def test_lsq_complex_poly_apply(degree, prec):
    # q(A) v with the complex least-squares q of a non-symmetric contour,
    # against the oracle's basis recurrence on the same points
    pp = load()
    from tests.test_gpu_sign import MEDIUM
    L = _q2_handle(pp, MEDIUM)
    try:
        z = _skew_ellipse()
        L.set(prec)
        pp.pp_set_poly_lsq(L.h, degree, z)
        P, H = lsq.basis(z, degree + 1)
        al = lsq.coeffs(P, z ** -0.5)
        v = synth.spinor_field(MEDIUM, 13)
        yd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        pp.pp_poly_apply(L.h, dev(v), yd)
        ref = lsq.apply(L.q2, H, al, len(z), v)
        assert rel(host(yd), ref) < {"f64": 1e-10, "dw": 5e-10}[prec]
    finally:
        L.close()


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("degree", [4, 8])
def test_lsq_complex_sign_solve(degree, prec):
    # pp_build_poly(PP_LSQ_CONTOUR) on the complex Q^2: the closed contour around
    # the complex Ritz values (no symmetry), then sign(Q) b against the dense
    # sign function
    pp = load()
    from tests.test_gpu_sign import SMALL, reference
    b, xs = reference(SMALL, 0)
    L = _q2_handle(pp, SMALL)
    try:
        L.set(prec)
        pp.pp_build_poly(L.h, degree, pp.PP_LSQ_CONTOUR)
        kind, x, _ = pp.pp_get_poly_nodes(L.h)
        assert kind == pp.PP_LSQ_CONTOUR and len(x) == degree + 1
        assert np.any(np.abs(np.imag(x)) > 0)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=800, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), xs) < (1e-10 if prec == "f64" else 5e-10)
    finally:
        L.close()


def test_lsq_complex_nodes_off_the_real_symmetry():
    # the contour pp_build_poly builds for the complex operator has no symmetry
    # about the real axis: the Newton nodes of q (degree + 1 Leja points of the
    # contour) are not a conjugation-closed set, all in the right half-plane
    pp = load()
    from tests.test_gpu_sign import SMALL
    L = _q2_handle(pp, SMALL)
    try:
        L.set("f64")
        pp.pp_build_poly(L.h, 6, pp.PP_LSQ_CONTOUR)
        _, x, _ = pp.pp_get_poly_nodes(L.h)
        assert len(x) == 7 and np.all(np.real(x) > 0)
        xs = set(np.round(np.asarray(x), 9))
        assert any(np.round(np.conj(v), 9) not in xs for v in xs)
    finally:
        L.close()
