"""GPU parity of the FP32 kernels and of the mixed-precision solve
(PP_PREC_MIXED), through the C ABI, against the FP64 oracle.

Tolerances (relative 2-norm):
* one operator application in FP32: 4e-7 (input rounding plus a handful of
  FP32 roundings of values of size |A||x|, |A||x| / |Ax| <= 2 here);
* q(A) v in FP32 by the Clenshaw recurrence: 1e-7 (deg + 1), about one FP32
  rounding per step carried by Clenshaw vectors of the size of q(A) v;
* mixed solves: the FP32 phase starts only once its rounding, amplified by
  kappa_pre, is below tol for the rest of the iteration, so the error must
  stay within max(3 x the error of the double-word solve at the same tol,
  tol): the stopping estimate lags the error by the same amount in both.
"""
import numpy as np
import pytest

import synth
from oracle import chebyshev as cheb, exact, operators as ops
from tests.libpp import load
from tests.test_gpu_parity import CASES, CASES_EVEN, Problem, dev, host, rel, set_prec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS_ALL = {"f64": 0, "dw": 1, "mixed": 2}


def set_p(pp, h, prec, side=0):
    o = pp.pp_default_opts()
    o.precision = PRECS_ALL[prec]
    o.side = side
    pp.pp_set_opts(h, o)


IDS = lambda c: f"{c[0]}{c[1]}{'csr' if c[3] else ''}"

_EXACT = {}


def exact_cached(P, b, power, key):
    if key not in _EXACT:
        _EXACT[key] = P.exact(b, power)
    return _EXACT[key]


@pytest.mark.parametrize("case", CASES + CASES_EVEN, ids=IDS)
def test_f32_op_apply(case):
    pp = load()
    P = Problem(pp, case[0], case[1], case[2], case[3])
    try:
        set_p(pp, P.h, "mixed")
        x = synth.rhs(P.n, 11)
        yd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_op_apply(P.h, dev(x), yd)
        assert rel(host(yd), P.A @ x) < 4e-7
    finally:
        P.close()


@pytest.mark.parametrize("degree", [0, 3, 8, 17])
@pytest.mark.parametrize("case", CASES[:3] + CASES[4:] + CASES_EVEN, ids=IDS)
def test_f32_poly_apply(case, degree):
    pp = load()
    P = Problem(pp, case[0], case[1], case[2], case[3], degree=degree)
    try:
        set_p(pp, P.h, "mixed")
        x = synth.rhs(P.n, 12)
        yd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(P.h, dev(x), yd)
        ref = cheb.q_apply(P.A.dot, P.coef, P.ab[0], P.ab[1], x)
        assert rel(host(yd), ref) < 1e-7 * (degree + 1)
    finally:
        P.close()


@pytest.mark.parametrize("tol", [1e-8, 1e-10])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
@pytest.mark.parametrize("degree", [4, 16])
@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3], CASES_EVEN[1]], ids=IDS)
def test_mixed_solve(case, degree, side, f, tol):
    pp = load()
    P = Problem(pp, case[0], case[1], case[2], case[3], degree=degree)
    try:
        b = synth.rhs(P.n, 0)
        bd, xd = dev(b), torch.empty(P.n, dtype=torch.float64, device="cuda")
        xs = exact_cached(P, b, 0.5 * f, (case, f))
        set_p(pp, P.h, "dw", side)
        st = pp.pp_apply(P.h, f, bd, xd, m_max=600, tol=tol)
        err_dw = rel(host(xd), xs)
        set_p(pp, P.h, "mixed", side)
        st = pp.pp_apply(P.h, f, bd, xd, m_max=600, tol=tol)
        assert st.status == pp.PP_OK
        err = rel(host(xd), xs)
        assert err <= max(3.0 * err_dw, tol), (err, err_dw, st.switch_iter)
    finally:
        P.close()


def test_mixed_switches_on_well_conditioned_problem():
    # kappa_pre ~ 1.2: the FP32 phase starts early and carries most steps
    # (checks every 2 steps: the default 64 / 17 = 3 leaves no check between
    # the first one and convergence on this small grid)
    pp = load()
    P = Problem(pp, "convdiff", (32, 18, 21), ch=0.5, degree=16)
    try:
        b = synth.rhs(P.n, 0)
        xd = torch.empty(P.n, dtype=torch.float64, device="cuda")
        set_p(pp, P.h, "mixed")
        o = pp.pp_default_opts()
        o.precision = pp.PP_PREC_MIXED
        o.check_every = 2
        pp.pp_set_opts(P.h, o)
        st = pp.pp_apply(P.h, 1, dev(b), xd, m_max=200, tol=1e-10)
        assert st.status == pp.PP_OK and 0 < st.switch_iter < st.iters
        assert rel(host(xd), P.exact(b, 0.5)) < 1e-10
        set_p(pp, P.h, "dw")
        st = pp.pp_apply(P.h, 1, dev(b), xd, m_max=200, tol=1e-10)
        assert st.switch_iter == 0
    finally:
        P.close()


def test_mixed_full_size_laplace2048():
    # 2D Laplacian 2048^2 (n = 4.2M), f = A^{-1/2}, degree 16, closed-form oracle;
    # the 1e-8 target is met with the estimate's tolerance one decade lower
    pp = load()
    dims = (2048, 2048)
    n = dims[0] * dims[1]
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    try:
        pp.pp_build_poly(h, 16)
        b = synth.rhs(n, 0)
        xs = exact.separable_fun(dims, b, -0.5)
        bd, xd = dev(b), torch.empty(n, dtype=torch.float64, device="cuda")
        for prec in ("mixed", "dw"):
            set_p(pp, h, prec)
            st = pp.pp_apply(h, -1, bd, xd, m_max=1000, tol=1e-9)
            assert st.status == pp.PP_OK
            assert rel(host(xd), xs) < 1e-8, prec
    finally:
        pp.pp_destroy(h)


def test_mixed_full_size_convdiff128():
    # 128^3 convection-diffusion, A^{1/2} b: mixed against a tight double-word solve
    pp = load()
    dims = (128, 128, 128)
    n = 128 ** 3
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 16)
        b = synth.rhs(n, 0)
        bd = dev(b)
        xr = torch.empty(n, dtype=torch.float64, device="cuda")
        xm = torch.empty_like(xr)
        set_p(pp, h, "dw")
        pp.pp_apply(h, 1, bd, xr, m_max=200, tol=1e-13)
        set_p(pp, h, "mixed")
        st = pp.pp_apply(h, 1, bd, xm, m_max=200, tol=1e-10)
        assert st.status == pp.PP_OK and st.switch_iter > 0
        assert rel(host(xm), host(xr)) < 1e-10
        # (A^{1/2})^2 b = A b in the mixed arithmetic
        ab = ops.convdiff(dims, 0.5) @ b
        x2 = torch.empty_like(xr)
        pp.pp_apply(h, 1, xm, x2, m_max=200, tol=1e-10)
        assert rel(host(x2), ab) < 1e-10
    finally:
        pp.pp_destroy(h)
