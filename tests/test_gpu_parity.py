"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative 2-norm): one operator application 1e-14 (FP64) /
2e-13 (double-word); q(A) v 1e-12 / 5e-12; full solves 1e-10 against the
exact solution for both arithmetics (the stated FP64 target).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import chebyshev as cheb, exact, krylov, operators as ops
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = {"f64": 0, "dw": 1}
OP_TOL = {"f64": 1e-14, "dw": 2e-13}
POLY_TOL = {"f64": 1e-12, "dw": 5e-12}
SOLVE_TOL = 1e-10


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def set_prec(pp, h, prec, side=0, orth=0, check_every=0, clenshaw=0):
    o = pp.pp_default_opts()
    o.precision = PRECS[prec]
    o.side = side
    o.orth = orth
    o.check_every = check_every
    o.clenshaw = clenshaw
    pp.pp_set_opts(h, o)


class Problem:
    """A test operator both as a library handle and as an oracle matrix."""

    def __init__(self, pp, kind, dims, ch=0.0, csr=False, degree=8):
        self.pp, self.kind, self.dims, self.ch = pp, kind, tuple(dims), ch
        self.n = int(np.prod(dims))
        if kind == "laplace":
            self.A = ops.laplace(self.dims)
            self.ab = ops.laplace_interval(self.dims)
        else:
            self.A = ops.convdiff(self.dims, ch)
            self.ab = ops.convdiff_interval(self.dims, ch)
        self.hermitian = kind == "laplace"
        self.keep = []
        if csr:
            skind = {2: "laplace2d5", 3: "laplace3d7"}[len(dims)] if kind == "laplace" else "convdiff3d7"
            rp, col, val = synth.stencil_csr(skind, self.dims, ch)
            self.keep = [dev(rp), dev(col), dev(val)]
            self.h = pp.pp_create_csr(self.n, *self.keep, is_hermitian=self.hermitian)
            self.interval = self.ab
        else:
            sk = {("laplace", 2): pp.PP_LAPLACE2D5, ("laplace", 3): pp.PP_LAPLACE3D7,
                  ("convdiff", 3): pp.PP_CONVDIFF3D7_UPWIND}[(kind, len(dims))]
            self.h = pp.pp_create_stencil(sk, self.dims, [ch] if kind == "convdiff" else None)
            self.interval = None
        self.build(degree)

    def build(self, degree):
        self.degree = degree
        self.pp.pp_build_poly(self.h, degree, interval_ab=self.interval)
        self.coef = cheb.interp_coeffs(self.ab[0], self.ab[1], degree + 1)

    def exact(self, b, power):
        if self.kind == "laplace":
            return exact.separable_fun(self.dims, b, power)
        if self.n <= 2000:
            return exact.dense_fun(self.A, b, power, hermitian=False)
        return krylov.plain_reference(self.A.dot, b, power, tol=1e-13, m_max=1500, k_chk=8)["x"]

    def close(self):
        self.pp.pp_destroy(self.h)


CASES = [("laplace", (61, 37), 0.0, False), ("laplace", (33, 17, 29), 0.0, False),
         ("convdiff", (33, 17, 29), 0.5, False), ("laplace", (61, 37), 0.0, True),
         ("convdiff", (19, 23, 9), 0.5, True)]
# even row lengths: the stencil kernels take the vector-load path (nx a
# multiple of the entries per 16-byte access); the cases above take the
# scalar path
CASES_EVEN = [("laplace", (64, 38), 0.0, False), ("convdiff", (32, 18, 21), 0.5, False)]


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("case", CASES + CASES_EVEN, ids=lambda c: f"{c[0]}{c[1]}{'csr' if c[3] else ''}")
def test_op_apply(case, prec):
    pp = load()
    P = Problem(pp, case[0], case[1], case[2], case[3])
    try:
        set_prec(pp, P.h, prec)
        x = synth.rhs(P.n, 11)
        xd, yd = dev(x), torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_op_apply(P.h, xd, yd)
        assert rel(host(yd), P.A @ x) < OP_TOL[prec]
    finally:
        P.close()


@pytest.mark.parametrize("scheme", ["horner", "clenshaw"])
@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("degree", [0, 1, 2, 3, 8, 17, 64])
@pytest.mark.parametrize("case", CASES[:3] + CASES[4:] + CASES_EVEN,
                         ids=lambda c: f"{c[0]}{c[1]}{'csr' if c[3] else ''}")
def test_poly_apply(case, degree, prec, scheme):
    # the Chebyshev interpolant by either evaluation scheme against the
    # oracle's three-term recurrence
    pp = load()
    P = Problem(pp, case[0], case[1], case[2], case[3], degree=degree)
    try:
        set_prec(pp, P.h, prec, clenshaw=int(scheme == "clenshaw"))
        x = synth.rhs(P.n, 12)
        xd, yd = dev(x), torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(P.h, xd, yd)
        ref = cheb.q_apply(P.A.dot, P.coef, P.ab[0], P.ab[1], x)
        # the non-normal convection-diffusion operator amplifies rounding in
        # any degree-64 evaluation, the oracle's three-term recurrence
        # included (both schemes land 2e-11 .. 5e-11 from it); Laplacians keep
        # the tight bound
        tol = POLY_TOL[prec] * (100.0 if case[0] == "convdiff" and degree > 17 else 1.0)
        assert rel(host(yd), ref) < tol
    finally:
        P.close()


@pytest.mark.parametrize("scheme", ["horner", "clenshaw"])
@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
@pytest.mark.parametrize("degree", [0, 4, 9])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2], CASES[3], CASES_EVEN[1]],
                         ids=lambda c: f"{c[0]}{c[1]}{'csr' if c[3] else ''}")
def test_solve_parity(case, degree, side, f, prec, scheme):
    pp = load()
    P = Problem(pp, case[0], case[1], case[2], case[3], degree=degree)
    try:
        set_prec(pp, P.h, prec, side=side, clenshaw=int(scheme == "clenshaw"))
        b = synth.rhs(P.n, 0)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, f, bd, xd, m_max=600, tol=1e-12)
        assert st.status == pp.PP_OK
        xs = P.exact(b, 0.5 * f)
        assert rel(host(xd), xs) < SOLVE_TOL
        # counters as in Table 1: 2d - 1 mvms per iteration plus start-up products
        extra = (degree if side == 0 else 0) + (1 if f == 1 else 0)
        assert st.mvms == st.iters * (2 * degree + 1) + extra
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
def test_misaligned_vectors_take_scalar_path(prec):
    # device vectors offset by one entry (8-byte aligned only): same result
    pp = load()
    P = Problem(pp, *CASES_EVEN[1], degree=5)
    try:
        set_prec(pp, P.h, prec)
        x = synth.rhs(P.n, 13)
        base = torch.zeros(P.n + 1, dtype=torch.float64, device="cuda")
        base[1:] = dev(x)
        out = torch.zeros(P.n + 1, dtype=torch.float64, device="cuda")
        pp.pp_op_apply(P.h, base[1:], out[1:])
        assert rel(host(out)[1:], P.A @ x) < OP_TOL[prec]
        pp.pp_poly_apply(P.h, base[1:], out[1:])
        ref = cheb.q_apply(P.A.dot, P.coef, P.ab[0], P.ab[1], x)
        assert rel(host(out)[1:], ref) < POLY_TOL[prec]
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
def test_iterations_match_oracle(prec):
    # same stopping rule as Algorithm 1 with checks every 64/d iterations
    pp = load()
    dims = (64, 64)
    P = Problem(pp, "laplace", dims, degree=8, csr=True)
    try:
        set_prec(pp, P.h, prec)
        b = synth.rhs(P.n, 0)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, -1, bd, xd, m_max=300, tol=1e-10)
        r = krylov.pp_arnoldi(P.A.dot, b, -0.5, P.coef, P.ab, side="left", m_max=300, tol=1e-10,
                              k_chk=64 // 9, hermitian=True, orth="lanczos")
        assert st.iters == r["iters"]
        assert st.inner_products == r["inner_products"]
        assert rel(host(xd), exact.separable_fun(dims, b, -0.5)) < SOLVE_TOL
    finally:
        P.close()


def test_degree_zero_equals_plain():
    # q constant: same iterate as plain (unpreconditioned) Lanczos from the oracle
    pp = load()
    P = Problem(pp, "laplace", (40, 30), degree=0)
    try:
        b = synth.rhs(P.n, 3)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        set_prec(pp, P.h, "f64", check_every=1)
        st = pp.pp_apply(P.h, -1, bd, xd, m_max=30, tol=0.0)
        assert st.status == pp.PP_ERR_NOT_CONVERGED and st.iters == 30
        r = krylov.pp_arnoldi(P.A.dot, b, -0.5, (1.0,), m_max=30, tol=0.0, k_chk=1, hermitian=True,
                              orth="lanczos")
        assert rel(host(xd), r["x"]) < 1e-11
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
def test_cgs2_on_hermitian_equals_lanczos(prec):
    pp = load()
    P = Problem(pp, "laplace", (20, 21, 22), degree=6)
    try:
        b = synth.rhs(P.n, 5)
        bd = dev(b)
        x1 = torch.empty(P.n, dtype=torch.float64, device="cuda")
        x2 = torch.empty_like(x1)
        set_prec(pp, P.h, prec, orth=1)
        pp.pp_apply(P.h, -1, bd, x1, m_max=200, tol=1e-12)
        set_prec(pp, P.h, prec, orth=2)
        st = pp.pp_apply(P.h, -1, bd, x2, m_max=200, tol=1e-12)
        m = st.iters
        assert st.inner_products == m * (m + 1) + m
        xs = P.exact(b, -0.5)
        assert rel(host(x1), xs) < SOLVE_TOL and rel(host(x2), xs) < SOLVE_TOL
    finally:
        P.close()


def test_identities_at_full_size_convdiff():
    # 3D convection-diffusion 128^3 (n = 2.1M): (A^{1/2})^2 b = A b and A^{-1/2} A^{1/2} b = b
    pp = load()
    dims = (128, 128, 128)
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 16)
        n = 128 ** 3
        b = synth.rhs(n, 0)
        A = ops.convdiff(dims, 0.5)
        for prec in ("dw", "f64"):
            set_prec(pp, h, prec)
            bd = dev(b)
            s1 = torch.empty(n, dtype=torch.float64, device="cuda")
            s2 = torch.empty_like(s1)
            st = pp.pp_apply(h, 1, bd, s1, m_max=100, tol=1e-12)
            assert st.status == pp.PP_OK
            pp.pp_apply(h, 1, s1, s2, m_max=100, tol=1e-12)
            assert rel(host(s2), A @ b) < SOLVE_TOL
            pp.pp_apply(h, -1, s1, s2, m_max=100, tol=1e-12)
            assert rel(host(s2), b) < SOLVE_TOL
    finally:
        pp.pp_destroy(h)


def test_edge_cases():
    pp = load()
    # n = 1
    h = pp.pp_create_stencil(pp.PP_LAPLACE3D7, (1, 1, 1))
    try:
        pp.pp_build_poly(h, 0, interval_ab=(5.0, 7.0))
        bd = dev(np.array([2.0]))
        xd = torch.empty(1, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, -1, bd, xd, m_max=5, tol=1e-12)
        assert abs(host(xd)[0] - 2.0 / np.sqrt(6.0)) < 1e-14 and st.breakdown == 1 and st.iters == 1
        st = pp.pp_apply(h, 1, bd, xd, m_max=5, tol=1e-12)
        assert abs(host(xd)[0] - 2.0 * np.sqrt(6.0)) < 1e-13
    finally:
        pp.pp_destroy(h)
    P = Problem(pp, "laplace", (17, 9), degree=3)
    try:
        n = P.n
        xd = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(P.h, -1, torch.zeros(n, dtype=torch.float64, device="cuda"), xd)
        assert st.status == pp.PP_OK and st.iters == 0 and float(xd.abs().max()) == 0.0
        bad = synth.rhs(n, 1)
        bad[5] = np.nan
        with pytest.raises(pp.PPError) as e:
            pp.pp_apply(P.h, -1, dev(bad), xd)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        b = synth.rhs(n, 2)
        st = pp.pp_apply(P.h, -1, dev(b), xd, m_max=2, tol=1e-14)
        assert st.status == pp.PP_ERR_NOT_CONVERGED and st.iters == 2
        assert np.all(np.isfinite(host(xd)))
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
def test_lucky_breakdown_diagonal_csr(prec):
    # P5: diagonal A with 12 distinct values -> exact after 12 steps (invariant space)
    pp = load()
    n = 3000
    a = np.repeat(np.linspace(1.0, 3.0, 12), n // 12)
    rp = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    keep = [dev(rp), dev(col), dev(a)]
    for orth in (1, 2):
        h = pp.pp_create_csr(n, *keep, is_hermitian=True)
        try:
            set_prec(pp, h, prec, orth=orth, check_every=1)
            pp.pp_build_poly(h, 2, interval_ab=(1.0, 3.0))
            b = synth.rhs(n, 4)
            xd = torch.empty(n, dtype=torch.float64, device="cuda")
            st = pp.pp_apply(h, -1, dev(b), xd, m_max=40, tol=1e-15)
            assert st.status == pp.PP_OK and st.iters <= 12
            assert rel(host(xd), a ** -0.5 * b) < 1e-11
        finally:
            pp.pp_destroy(h)


def test_apply_host_matches_device():
    pp = load()
    P = Problem(pp, "convdiff", (24, 20, 16), ch=0.5, degree=4)
    try:
        b = synth.rhs(P.n, 9)
        xh = np.empty(P.n)
        st = pp.pp_apply_host(P.h, 1, b, xh, m_max=100, tol=1e-12)
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_apply(P.h, 1, dev(b), xd, m_max=100, tol=1e-12)
        assert np.array_equal(xh, host(xd))  # deterministic reductions
        assert st.status == pp.PP_OK
    finally:
        P.close()
