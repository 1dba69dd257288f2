"""GPU parity of the Ritz / harmonic Ritz preconditioning polynomials (Sec. 5.2)
through the C ABI against the oracle (oracle/ritz.py).

* nodes: the library's node run (Arnoldi with CGS2 on A from the SplitMix64
  start vector) against the oracle's on the same start vector: the sorted
  nodes agree to 1e-10 relative to the largest; q agrees as a polynomial to
  1e-8 on [a,b] (its Leja order may differ at near-ties, q does not).
* the library's Newton coefficients give the same interpolant as the
  oracle's divided differences of the same nodes (1e-12 on [a,b]).
* q(A) v by the Horner chain against the oracle's term-by-term Newton sum
  with the library's own nodes: 1e-11 (FP64) / 5e-11 (double-word) /
  2e-7 (deg + 1) (FP32).
* solves: 1e-10 against the exact solution (FP64, double-word); mixed
  precision within max(3 x the double-word error, tol).
"""
import numpy as np
import pytest

import synth
from oracle import exact, krylov, operators as ops, ritz, wilson
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"f64": 0, "dw": 1, "mixed": 2}
M0 = 0.1


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def kind_of(pp, name):
    return {"ritz": pp.PP_RITZ_LEJA, "harmonic": pp.PP_HARMONIC_RITZ}[name]


class Problem:
    """Hermitian test operator as a library handle (stencil or CSR) and as a sparse matrix."""

    def __init__(self, pp, dims, csr=False, prec="f64", side=0, two_pass=False):
        self.pp, self.dims = pp, tuple(dims)
        self.n = int(np.prod(dims))
        self.A = ops.laplace(self.dims)
        self.keep = []
        if csr:
            rp, col, val = synth.stencil_csr({2: "laplace2d5", 3: "laplace3d7"}[len(dims)], self.dims)
            self.keep = [dev(rp), dev(col), dev(val)]
            self.h = pp.pp_create_csr(self.n, *self.keep, is_hermitian=True)
        else:
            sk = {2: pp.PP_LAPLACE2D5, 3: pp.PP_LAPLACE3D7}[len(dims)]
            self.h = pp.pp_create_stencil(sk, self.dims)
        self.set(prec, side, two_pass)

    def set(self, prec, side=0, two_pass=False):
        o = self.pp.pp_default_opts()
        o.precision = PREC[prec]
        o.side = side
        o.two_pass = 1 if two_pass else 0
        self.pp.pp_set_opts(self.h, o)

    def build(self, degree, kind):
        self.pp.pp_build_poly(self.h, degree, kind_of(self.pp, kind))
        k, self.x, self.cap = self.pp.pp_get_poly_nodes(self.h)
        assert k == kind_of(self.pp, kind)
        self.a, self.ab, self.img = self.pp.pp_get_poly(self.h)

    def close(self):
        self.pp.pp_destroy(self.h)


CASES = [((61, 37), False), ((17, 13, 11), False), ((45, 31), True), ((64, 38), False)]
IDS = ["lap2d", "lap3d", "lap2dcsr", "lap2d_even"]


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("kind", ["ritz", "harmonic"])
@pytest.mark.parametrize("degree", [0, 1, 4, 9, 24])
@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_nodes_match_oracle(case, degree, kind, prec):
    pp = load()
    P = Problem(pp, case[0], case[1], prec)
    try:
        P.build(degree, kind)
        xo, ao = ritz.ritz_poly(P.A.dot, P.n, degree, harmonic=(kind == "harmonic"))
        assert len(P.x) == degree + 1 and len(P.a) == degree + 1
        scale = np.abs(xo).max()
        assert np.abs(np.sort(P.x) - np.sort(xo)).max() < 1e-10 * scale
        # the library's order reversed is a Leja order of its nodes (greedy maximum, to rounding)
        xl = P.x[::-1]
        assert xl[0] == np.abs(xl).max()
        for k in range(1, len(xl)):
            prods = [np.prod(np.abs(z - xl[:k])) for z in xl[k:]]
            assert np.prod(np.abs(xl[k] - xl[:k])) >= max(prods) * (1 - 1e-9)
        # Newton coefficients = divided differences of the library's nodes: the
        # same interpolant (the high-order coefficients carry the rounding of
        # z^{-1/2} at the nodes amplified by the divided differences, so the
        # polynomial is compared, and the interpolation conditions)
        z = np.linspace(P.ab[0], P.ab[1], 257)
        an = ritz.newton_coeffs(P.x)
        assert rel(ritz.newton_eval(P.a, P.x, z), ritz.newton_eval(an, P.x, z)) < 1e-12
        assert np.allclose(P.a[:3], an[:3], rtol=1e-12)
        assert np.allclose(ritz.newton_eval(P.a, P.x, P.x), P.x ** -0.5, rtol=1e-10)
        # the same polynomial as the oracle's
        assert rel(ritz.newton_eval(P.a, P.x, z), ritz.newton_eval(ao, xo, z)) < 1e-8
        # positivity and the image interval of z q(z)^2 on [a,b]
        zz = np.geomspace(P.ab[0], P.ab[1], 4001)
        q = ritz.newton_eval(P.a, P.x, zz)
        assert q.min() > 0
        p = zz * q * q
        assert P.img[0] <= p.min() * (1 + 1e-9) and P.img[1] >= p.max() * (1 - 1e-9)
        if case[1]:  # CSR: the extreme Ritz values of the node run, widened
            if kind == "ritz":
                assert P.ab == pytest.approx((0.95 * P.x.min(), 1.01 * P.x.max()), rel=1e-14)
            assert 0 < P.ab[0] < P.ab[1]
        else:        # stencils: the closed-form spectral interval
            lam = exact.separable_eigs(P.dims)
            assert (P.ab[0], P.ab[1]) == pytest.approx((lam.min(), lam.max()), rel=1e-12)
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("degree", [0, 1, 2, 3, 8, 17])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_poly_apply_horner(case, degree, prec):
    pp = load()
    P = Problem(pp, case[0], case[1], "dw" if prec == "mixed" else prec)
    try:
        P.build(degree, "ritz")
        P.set(prec)
        v = synth.rhs(P.n, 12)
        yd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(P.h, dev(v), yd)
        ref = ritz.newton_apply(P.A.dot, P.a, P.x, v)
        tol = {"f64": 1e-11, "dw": 5e-11, "mixed": 2e-7 * (degree + 1)}[prec]
        assert rel(host(yd), ref) < tol
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
@pytest.mark.parametrize("kind", ["ritz", "harmonic"])
@pytest.mark.parametrize("degree", [4, 12])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2]], ids=IDS[:3])
def test_solve_ritz(case, degree, kind, side, f, prec):
    pp = load()
    P = Problem(pp, case[0], case[1], "dw" if prec == "mixed" else prec, side)
    try:
        P.build(degree, kind)
        b = synth.rhs(P.n, 0)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        xs = exact.separable_fun(P.dims, b, 0.5 * f)
        tol = 1e-12
        if prec == "mixed":
            P.set("dw", side)
            pp.pp_apply(P.h, f, bd, xd, m_max=600, tol=tol)
            err_dw = rel(host(xd), xs)
            P.set("mixed", side)
        st = pp.pp_apply(P.h, f, bd, xd, m_max=600, tol=tol)
        assert st.status == pp.PP_OK
        err = rel(host(xd), xs)
        if prec == "mixed":
            assert err <= max(3.0 * err_dw, tol), (err, err_dw)
        else:
            assert err < 1e-10
        extra = (degree if side == 0 else 0) + (1 if f == 1 else 0)
        assert st.mvms == st.iters * (2 * degree + 1) + extra
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("kind", ["ritz", "harmonic"])
def test_iterations_match_oracle(kind, prec):
    # Algorithm 1 in the oracle with the library's own q (same nodes and
    # coefficients): the same stopping checks, so the same iteration count
    pp = load()
    dims = (64, 64)
    P = Problem(pp, dims, True, prec)
    try:
        deg = 8
        P.build(deg, kind)
        b = synth.rhs(P.n, 0)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, -1, bd, xd, m_max=300, tol=1e-10)
        r = krylov.pp_arnoldi(P.A.dot, b, -0.5, q=(deg, lambda v: ritz.newton_apply(P.A.dot, P.a, P.x, v)),
                              side="left", m_max=300, tol=1e-10, k_chk=64 // (deg + 1), hermitian=True,
                              orth="lanczos")
        assert st.iters == r["iters"]
        assert rel(host(xd), r["x"]) < 1e-9
        assert rel(host(xd), exact.separable_fun(dims, b, -0.5)) < 1e-9
    finally:
        P.close()


def test_ritz_beats_plain_lanczos():
    # Sec. 5.2 / Example 2: interpolation at Ritz values lowers the iteration count
    pp = load()
    P = Problem(pp, (128, 96), False, "dw")
    try:
        b = synth.rhs(P.n, 0)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        P.build(0, "ritz")
        st0 = pp.pp_apply(P.h, -1, bd, xd, m_max=1000, tol=1e-10)
        P.build(16, "ritz")
        st1 = pp.pp_apply(P.h, -1, bd, xd, m_max=1000, tol=1e-10)
        assert st0.status == pp.PP_OK and st1.status == pp.PP_OK
        assert st1.iters * 4 < st0.iters
        assert rel(host(xd), exact.separable_fun(P.dims, b, -0.5)) < 1e-9
    finally:
        P.close()


def test_small_n_reduces_degree():
    # n = 6 points: the Krylov space of any start vector has dimension <= 6,
    # so a degree-10 request gets at most 6 nodes
    pp = load()
    P = Problem(pp, (3, 2), False, "f64")
    try:
        P.build(10, "ritz")
        lam = np.sort(exact.separable_eigs(P.dims))
        assert 1 <= len(P.x) <= 6 and len(P.a) == len(P.x)
        xo, _ = ritz.ritz_poly(P.A.dot, P.n, 10)
        assert len(xo) == len(P.x)
        assert np.allclose(np.sort(P.x), np.sort(xo), rtol=1e-10)
        # every node is an eigenvalue of A (the space is invariant)
        assert all(np.abs(lam - x).min() < 1e-10 * lam.max() for x in P.x)
        b = synth.rhs(P.n, 1)
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, -1, dev(b), xd, m_max=20, tol=1e-13)
        assert st.status == pp.PP_OK
        assert rel(host(xd), exact.dense_fun(P.A.toarray(), b, -0.5, hermitian=True)) < 1e-11
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("kind", ["ritz", "harmonic"])
def test_wilson_ritz(kind, prec):
    # Example 2 builds q from Ritz values of the Hermitian positive definite
    # operator; here A = D^H D on a small random-link lattice
    pp = load()
    dims = (2, 3, 2, 4)
    links = synth.wilson_links(dims, 1)
    A = wilson.dhd_matrix(dims, links, M0)
    V = int(np.prod(dims))
    n = 12 * V
    links_d = dev(links.astype(np.complex64))
    h = pp.pp_create_stencil(pp.PP_WILSON4D_DHD, dims, [M0], links=links_d, dtype=pp.PP_C128)
    try:
        o = pp.pp_default_opts()
        o.precision = PREC["dw" if prec == "mixed" else prec]
        pp.pp_set_opts(h, o)
        deg = 6
        pp.pp_build_poly(h, deg, kind_of(pp, kind))
        _, x, _ = pp.pp_get_poly_nodes(h)
        a, ab, _ = pp.pp_get_poly(h)
        xo, _ = ritz.ritz_poly(A.dot, n, deg, harmonic=(kind == "harmonic"), complex_=True)
        assert np.abs(np.sort(x) - np.sort(xo)).max() < 1e-10 * np.abs(xo).max()
        b = synth.spinor_field(dims, 0)
        xs = exact.dense_fun(A, b, -0.5, hermitian=True)
        xd = torch.empty(n, dtype=torch.complex128, device="cuda")
        o.precision = PREC[prec]
        pp.pp_set_opts(h, o)
        v = synth.spinor_field(dims, 5)
        pp.pp_poly_apply(h, dev(v), xd)
        ptol = {"f64": 1e-11, "dw": 5e-11, "mixed": 2e-7 * (deg + 1)}[prec]
        assert rel(host(xd), ritz.newton_apply(A.dot, a, x, v)) < ptol
        st = pp.pp_apply(h, -1, dev(b), xd, m_max=400, tol=1e-11)
        assert st.status == pp.PP_OK
        assert rel(host(xd), xs) < (1e-10 if prec != "mixed" else 1e-8)
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["dw", "mixed"])
def test_batch_mixes_ritz_and_chebyshev(prec):
    # a Ritz and a Chebyshev handle of the same degree run in separate groups;
    # each process gives what pp_apply gives it alone
    pp = load()
    probs = [((48, 40), "ritz", 6), ((48, 40), "cheb", 6), ((13, 11, 9), "harmonic", 4), ((30, 50), "ritz", 0)]
    hs, bs, xs, xs1, ref = [], [], [], [], []
    try:
        for i, (dims, kind, deg) in enumerate(probs):
            sk = {2: pp.PP_LAPLACE2D5, 3: pp.PP_LAPLACE3D7}[len(dims)]
            h = pp.pp_create_stencil(sk, dims)
            o = pp.pp_default_opts()
            o.precision = PREC["dw"]
            pp.pp_set_opts(h, o)
            pp.pp_build_poly(h, deg, pp.PP_CHEBYSHEV if kind == "cheb" else kind_of(pp, kind))
            o.precision = PREC[prec]
            pp.pp_set_opts(h, o)
            hs.append(h)
            n = int(np.prod(dims))
            b = synth.rhs(n, 20 + i)
            bs.append(dev(b))
            xs.append(torch.empty(n, dtype=torch.float64, device="cuda"))
            xs1.append(torch.empty(n, dtype=torch.float64, device="cuda"))
            ref.append(exact.separable_fun(dims, b, -0.5))
        sts = pp.pp_apply_batch(hs, [-1] * len(hs), bs, xs, m_max=600, tol=1e-11)
        for i, h in enumerate(hs):
            assert sts[i].status == pp.PP_OK
            st = pp.pp_apply(h, -1, bs[i], xs1[i], m_max=600, tol=1e-11)
            assert st.iters == sts[i].iters
            got = host(xs[i])
            assert rel(got, host(xs1[i])) < (1e-14 if prec == "dw" else 1e-6)
            assert rel(got, ref[i]) < (1e-10 if prec == "dw" else 1e-8)
    finally:
        for h in hs:
            pp.pp_destroy(h)


def test_two_pass_with_ritz():
    pp = load()
    P = Problem(pp, (61, 37), False, "dw")
    try:
        P.build(8, "harmonic")
        b = synth.rhs(P.n, 0)
        bd = dev(b)
        x1 = torch.empty(P.n, dtype=torch.float64, device="cuda")
        x2 = torch.empty(P.n, dtype=torch.float64, device="cuda")
        s1 = pp.pp_apply(P.h, 1, bd, x1, m_max=400, tol=1e-12)
        P.set("dw", two_pass=True)
        s2 = pp.pp_apply(P.h, 1, bd, x2, m_max=400, tol=1e-12)
        assert s1.status == pp.PP_OK and s2.status == pp.PP_OK and s1.iters == s2.iters
        assert rel(host(x2), host(x1)) < 1e-13
        assert rel(host(x2), exact.separable_fun(P.dims, b, 0.5)) < 1e-10
    finally:
        P.close()


def test_static_apply_with_ritz():
    pp = load()
    P = Problem(pp, (40, 30), False, "f64")
    try:
        P.build(7, "ritz")
        v = synth.rhs(P.n, 3)
        y1 = torch.empty(P.n, dtype=torch.float64, device="cuda")
        y2 = torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(P.h, dev(v), y1)
        pp.pp_poly_apply_static(P.h, dev(v), y2)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
        assert rel(host(y2), ritz.newton_apply(P.A.dot, P.a, P.x, v)) < 1e-11
    finally:
        P.close()


# ---- non-Hermitian operators: Arnoldi Ritz values, conjugate pairs ----

def same_set(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    return len(a) == len(b) and max(np.abs(b - z).min() for z in a) < tol and \
        max(np.abs(a - z).min() for z in b) < tol


def paired_nodes(a, b, deg):
    """deg + 1 nodes in [a, b]: the first-kind Chebyshev nodes with some
    neighbouring couples replaced by a conjugate pair at their mean."""
    d = deg + 1
    t = np.pi * (np.arange(d) + 0.5) / d
    z = list(0.5 * (a + b) + 0.5 * (b - a) * np.cos(t))
    out, i = [], 0
    while i < d:
        if i + 1 < d and i % 4 == 1:
            m, w = 0.5 * (z[i] + z[i + 1]), 0.25 * abs(z[i] - z[i + 1])
            out += [m + 1j * w, m - 1j * w]
            i += 2
        else:
            out.append(complex(z[i]))
            i += 1
    return np.array(out)


class NonHerm:
    """Upwind convection-diffusion (real, non-symmetric) as stencil or CSR handle."""

    def __init__(self, pp, dims, csr, prec):
        self.pp, self.dims = pp, tuple(dims)
        self.n = int(np.prod(dims))
        self.A = ops.convdiff(self.dims, 0.5)
        self.ab = ops.convdiff_interval(self.dims, 0.5)
        self.keep = []
        if csr:
            rp, col, val = synth.stencil_csr("convdiff3d7", self.dims, 0.5)
            self.keep = [dev(rp), dev(col), dev(val)]
            self.h = pp.pp_create_csr(self.n, *self.keep, is_hermitian=False)
        else:
            self.h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, self.dims, [0.5])
        self.set(prec)

    def set(self, prec, side=0):
        o = self.pp.pp_default_opts()
        o.precision = PREC[prec]
        o.side = side
        self.pp.pp_set_opts(self.h, o)

    def close(self):
        self.pp.pp_destroy(self.h)


NH_CASES = [((13, 11, 9), False), ((9, 8, 7), True), ((16, 10, 6), False)]
NH_IDS = ["cd_stencil", "cd_csr", "cd_even"]


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("degree", [1, 4, 8, 16])
@pytest.mark.parametrize("case", NH_CASES, ids=NH_IDS)
def test_poly_apply_conjugate_pairs(case, degree, prec):
    # q at nodes with conjugate pairs: the real-basis chain (its pair steps read
    # w_{i+2} with the coefficient (Im x/cap)^2) against the oracle's complex
    # Newton sum at the library's own nodes
    pp = load()
    P = NonHerm(pp, case[0], case[1], prec)
    try:
        z = paired_nodes(*P.ab, degree)
        pp.pp_set_poly_nodes(P.h, z, interval_ab=P.ab)
        kind, x, _ = pp.pp_get_poly_nodes(P.h)
        assert kind == pp.PP_NODES
        v = synth.rhs(P.n, 7)
        yd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(P.h, dev(v), yd)
        ref = ritz.newton_apply(P.A.dot, ritz.newton_coeffs(x), x, v)
        tol = {"f64": 1e-11, "dw": 5e-11, "mixed": 2e-7 * (degree + 1)}[prec]
        assert rel(host(yd), ref) < tol
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("degree", [4, 12])
@pytest.mark.parametrize("case", NH_CASES[:2], ids=NH_IDS[:2])
def test_solve_conjugate_pairs(case, degree, f, prec):
    pp = load()
    P = NonHerm(pp, case[0], case[1], prec)
    try:
        pp.pp_set_poly_nodes(P.h, paired_nodes(*P.ab, degree))
        b = synth.rhs(P.n, 0)
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, f, dev(b), xd, m_max=400, tol=1e-12)
        assert st.status == pp.PP_OK
        xs = exact.dense_fun(P.A.toarray(), b, 0.5 * f, hermitian=False)
        assert rel(host(xd), xs) < 1e-10
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("kind", ["ritz", "harmonic"])
@pytest.mark.parametrize("degree", [1, 4, 8, 16])
@pytest.mark.parametrize("case", NH_CASES[:2], ids=NH_IDS[:2])
def test_nonhermitian_ritz(case, degree, kind, prec):
    # node run on a non-normal operator: Arnoldi (CGS2) + Francis QR of H_d
    # against the oracle's Arnoldi + LAPACK eigenvalues on the same start
    # vector (eigenvalues of a non-normal H_d move by more than its rounding:
    # 1e-7 relative); then the solve against the dense definition
    pp = load()
    P = NonHerm(pp, case[0], case[1], prec)
    try:
        pp.pp_build_poly(P.h, degree, kind_of(pp, kind))
        k, x, _ = pp.pp_get_poly_nodes(P.h)
        assert k == kind_of(pp, kind)
        xo, _ = ritz.ritz_poly(P.A.dot, P.n, degree, harmonic=(kind == "harmonic"), hermitian=False)
        assert same_set(x, xo, 1e-7 * np.abs(xo).max())
        assert np.all(np.real(x) > 0)
        b = synth.rhs(P.n, 0)
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, 1, dev(b), xd, m_max=400, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), exact.dense_fun(P.A.toarray(), b, 0.5, hermitian=False)) < 1e-10
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["dw", "mixed"])
def test_batch_conjugate_pairs(prec):
    # two convection-diffusion handles of the same degree in one batch group,
    # one with conjugate pairs (steps with a y term) and one with real nodes
    # (coefficient 0 on y in those steps): each equals its lone pp_apply
    pp = load()
    hs, bs, xs, x1 = [], [], [], []
    try:
        for i, paired in enumerate([True, False]):
            dims = (14, 12, 10)
            h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
            o = pp.pp_default_opts()
            o.precision = PREC[prec]
            pp.pp_set_opts(h, o)
            a, b = ops.convdiff_interval(dims, 0.5)
            z = paired_nodes(a, b, 8)
            if not paired:
                t = np.pi * (np.arange(9) + 0.5) / 9
                z = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(t)
            pp.pp_set_poly_nodes(h, z)
            hs.append(h)
            n = int(np.prod(dims))
            bs.append(dev(synth.rhs(n, 30 + i)))
            xs.append(torch.empty(n, dtype=torch.float64, device="cuda"))
            x1.append(torch.empty(n, dtype=torch.float64, device="cuda"))
        sts = pp.pp_apply_batch(hs, [1, -1], bs, xs, m_max=400, tol=1e-11)
        for i, h in enumerate(hs):
            assert sts[i].status == pp.PP_OK
            st = pp.pp_apply(h, [1, -1][i], bs[i], x1[i], m_max=400, tol=1e-11)
            assert st.iters == sts[i].iters
            assert rel(host(xs[i]), host(x1[i])) < (1e-14 if prec == "dw" else 1e-6)
    finally:
        for h in hs:
            pp.pp_destroy(h)
