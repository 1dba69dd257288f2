"""GPU parity of the Wilson D^H D operator path (PP_WILSON4D_DHD) through the
C ABI against the oracle (oracle/wilson.py).

Vectors are complex128 (12 components per site).  Tolerances (relative
2-norm): one application of A = D^H D 1e-13 (FP64 and double-word; two
stencil applications with 17 terms each) and 1e-6 in FP32; q(A) v 1e-12 /
5e-12 / 2e-7 (deg + 1); solves 1e-10 against the dense or Fourier closed form
(mixed: within max(3 x the double-word error, tol)).
"""
import numpy as np
import pytest

import synth
from oracle import chebyshev as cheb, exact, wilson
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"f64": 0, "dw": 1, "mixed": 2}
OP_TOL = {"f64": 1e-13, "dw": 1e-13, "mixed": 1e-6}
M0 = 0.1


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


class Lattice:
    def __init__(self, pp, dims, links, degree=8, interval=None):
        self.pp, self.dims = pp, tuple(dims)
        self.V = int(np.prod(dims))
        self.n = 12 * self.V
        self.links_d = dev(links.astype(np.complex64))
        self.h = pp.pp_create_stencil(pp.PP_WILSON4D_DHD, self.dims, [M0], links=self.links_d,
                                      dtype=pp.PP_C128)
        self.links = links
        self.A = None
        self.degree = degree
        if interval is not None or degree >= 0:
            pp.pp_build_poly(self.h, degree, interval_ab=interval)
            self.coef, self.ab, _ = pp.pp_get_poly(self.h)

    def matrix(self):
        if self.A is None:
            self.A = wilson.dhd_matrix(self.dims, self.links, M0)
        return self.A

    def set(self, prec, side=0, clenshaw=0):
        o = self.pp.pp_default_opts()
        o.precision = PREC[prec]
        o.side = side
        o.clenshaw = clenshaw
        self.pp.pp_set_opts(self.h, o)

    def close(self):
        self.pp.pp_destroy(self.h)


def small_interval(A):
    lam = np.linalg.eigvalsh(A.toarray())
    return float(lam[0]), float(lam[-1])


DIMS_SMALL = (2, 3, 2, 4)


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("dims", [DIMS_SMALL, (4, 4, 2, 6)])
def test_wilson_op_apply(dims, prec):
    pp = load()
    L = Lattice(pp, dims, synth.wilson_links(dims, 1), degree=0, interval=(0.01, 100.0))
    try:
        L.set(prec)
        x = synth.spinor_field(dims, 11)
        yd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        pp.pp_op_apply(L.h, dev(x), yd)
        assert rel(host(yd), L.matrix() @ x) < OP_TOL[prec]
    finally:
        L.close()


@pytest.mark.parametrize("scheme", ["horner", "clenshaw"])
@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("degree", [1, 2, 8])
def test_wilson_poly_apply(degree, prec, scheme):
    pp = load()
    dims = (4, 4, 2, 6)
    links = synth.wilson_links(dims, 1)
    A = wilson.dhd_matrix(dims, links, M0)
    L = Lattice(pp, dims, links, degree=degree, interval=(0.05, 60.0))
    try:
        L.set(prec, clenshaw=int(scheme == "clenshaw"))
        x = synth.spinor_field(dims, 12)
        yd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        pp.pp_poly_apply(L.h, dev(x), yd)
        ref = cheb.q_apply(A.dot, L.coef, 0.05, 60.0, x)
        tol = {"f64": 1e-12, "dw": 5e-12, "mixed": 2e-7 * (degree + 1)}[prec]
        assert rel(host(yd), ref) < tol
    finally:
        L.close()


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("degree", [0, 8])
def test_wilson_solve_small(degree, f, prec):
    pp = load()
    dims = DIMS_SMALL
    links = synth.wilson_links(dims, 1)
    A = wilson.dhd_matrix(dims, links, M0)
    lo, hi = small_interval(A)
    L = Lattice(pp, dims, links, degree=degree, interval=(lo, hi))
    try:
        b = synth.spinor_field(dims, 0)
        xs = exact.dense_fun(A, b, 0.5 * f, hermitian=True)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        L.set("dw")
        pp.pp_apply(L.h, f, dev(b), xd, m_max=400, tol=1e-11)
        err_dw = rel(host(xd), xs)
        L.set(prec)
        st = pp.pp_apply(L.h, f, dev(b), xd, m_max=400, tol=1e-11)
        assert st.status == pp.PP_OK
        err = rel(host(xd), xs)
        assert err < 1e-10 if prec != "mixed" else err <= max(3 * err_dw, 1e-11)
    finally:
        L.close()


def test_wilson_interval_estimate_encloses_spectrum():
    pp = load()
    dims = (4, 4, 2, 6)
    links = synth.wilson_links(dims, 1)
    lo, hi = small_interval(wilson.dhd_matrix(dims, links, M0))
    L = Lattice(pp, dims, links, degree=8)  # interval from the Lanczos estimate
    try:
        a, b = L.ab
        assert a <= lo and b >= hi
        assert a >= 0.5 * lo and b <= 1.5 * hi
    finally:
        L.close()


@pytest.mark.parametrize("prec", ["dw", "mixed"])
def test_wilson_free_field_full_size(prec):
    # 16^3 x 32 lattice (n = 1,572,864 complex), U = 1: Fourier closed form
    pp = load()
    dims = (16, 16, 16, 32)
    L = Lattice(pp, dims, synth.unit_links(dims), degree=16)
    try:
        a, b = L.ab
        lam = wilson.free_eigs(dims, M0)
        assert a <= lam.min() and b >= lam.max()
        L.set(prec)
        bv = synth.spinor_field(dims, 0)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, -1, dev(bv), xd, m_max=300, tol=1e-11)
        assert st.status == pp.PP_OK
        assert rel(host(xd), wilson.free_field_fun(dims, bv, -0.5, M0)) < 1e-10
    finally:
        L.close()


def test_wilson_identities_full_size():
    # random SU(3) links on 16^3 x 32: (A^{1/2})^2 b = A b and A^{-1/2} A^{1/2} b = b
    pp = load()
    dims = (16, 16, 16, 32)
    L = Lattice(pp, dims, synth.wilson_links(dims, 1), degree=16)
    try:
        n = L.n
        bv = dev(synth.spinor_field(dims, 0))
        ab = torch.empty(n, dtype=torch.complex128, device="cuda")
        s1, s2 = torch.empty_like(ab), torch.empty_like(ab)
        L.set("dw")
        pp.pp_op_apply(L.h, bv, ab)
        for prec in ("dw", "mixed"):
            L.set(prec)
            st = pp.pp_apply(L.h, 1, bv, s1, m_max=300, tol=1e-11)
            assert st.status == pp.PP_OK
            pp.pp_apply(L.h, 1, s1, s2, m_max=300, tol=1e-11)
            assert rel(host(s2), host(ab)) < 1e-10
            pp.pp_apply(L.h, -1, s1, s2, m_max=300, tol=1e-11)
            assert rel(host(s2), host(bv)) < 1e-10
    finally:
        L.close()


def exact_gauge(V, rng):
    """SU(3) matrices with entries in {0, +-1, +-i}: phase times permutation
    (exact in complex64, so U^G is exactly representable)."""
    perms = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]
    phases = np.array([1, 1j, -1, -1j])
    G = np.zeros((V, 3, 3), dtype=np.complex128)
    for s in range(V):
        p = perms[rng.integers(6)]
        P = np.zeros((3, 3))
        P[np.arange(3), p] = 1.0
        d1, d2 = phases[rng.integers(4)], phases[rng.integers(4)]
        d3 = 1.0 / (d1 * d2 * np.linalg.det(P))
        G[s] = np.diag([d1, d2, d3]) @ P
    return G


def test_wilson_gauge_covariance_gpu():
    # f(A[U^G]) G b = G f(A[U]) b for a random gauge transformation G
    pp = load()
    dims = (8, 8, 8, 8)
    U = synth.wilson_links(dims, 1).astype(np.complex128)
    G = exact_gauge(int(np.prod(dims)), np.random.default_rng(7))
    Ug = wilson.gauge_transform(dims, U, G)
    assert np.array_equal(Ug.astype(np.complex64).astype(np.complex128), Ug)
    b = synth.spinor_field(dims, 3)
    L1 = Lattice(pp, dims, U, degree=-1)
    L2 = Lattice(pp, dims, Ug, degree=-1)
    try:
        pp.pp_build_poly(L1.h, 8)
        _, ab, _ = pp.pp_get_poly(L1.h)
        pp.pp_build_poly(L2.h, 8, interval_ab=ab)
        x1 = torch.empty(L1.n, dtype=torch.complex128, device="cuda")
        x2 = torch.empty_like(x1)
        for L in (L1, L2):
            L.set("dw")
        pp.pp_apply(L1.h, -1, dev(b), x1, m_max=300, tol=1e-12)
        pp.pp_apply(L2.h, -1, dev(wilson.gauge_apply(G, b)), x2, m_max=300, tol=1e-12)
        assert rel(host(x2), wilson.gauge_apply(G, host(x1))) < 1e-10
    finally:
        L1.close()
        L2.close()
