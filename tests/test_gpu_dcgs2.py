"""GPU parity of Arnoldi with delayed reorthogonalization (PP_ORTH_DCGS2)
through the C ABI.

The delayed scheme applies A q(A)^2 to each new basis vector after its
first Gram-Schmidt pass and completes its second pass, its normalization
and the next vector's first pass from one sweep of inner products (pp.h).
In exact arithmetic it builds the same basis and H_m as CGS2, so the
stopping checks fall at the same Krylov dimensions: the tests compare
iteration counts and results with CGS2 (1e-12) and the results with the
FP64 oracle's closed form (1e-10 in FP64 and double-word; mixed precision
within max(3 x the double-word error, tol), as for CGS2), on odd sizes (a
ragged last chunk), the graph Laplacian of Example 3 (1e-7), a lucky
breakdown, and the refusals.
"""
import numpy as np
import pytest

import synth
from oracle import exact, operators as ops
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


def solve(pp, h, f, b, prec, orth, tol=1e-12, m_max=300, check_every=0):
    o = pp.pp_default_opts()
    o.precision = PREC[prec]
    o.orth = orth
    o.check_every = check_every
    pp.pp_set_opts(h, o)
    x = torch.empty(b.shape[0], dtype=torch.float64, device="cuda")
    st = pp.pp_apply(h, f, dev(b), x, m_max=m_max, tol=tol)
    return st, host(x)


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("f", [1, -1], ids=["sqrt", "invsqrt"])
@pytest.mark.parametrize("degree", [0, 4, 9])
def test_dcgs2_convdiff_against_cgs2_and_closed_form(degree, f, prec):
    pp = load()
    dims = (13, 11, 9)  # 1287 unknowns: a ragged last chunk
    n = int(np.prod(dims))
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, degree)
        b = synth.rhs(n, 21)
        xs = exact.separable_fun(dims, b, 0.5 * f, "convdiff", 0.5)
        s1, x1 = solve(pp, h, f, b, prec, pp.PP_ORTH_CGS2)
        s2, x2 = solve(pp, h, f, b, prec, pp.PP_ORTH_DCGS2)
        assert s1.status == pp.PP_OK and s2.status == pp.PP_OK
        assert s2.iters == s1.iters and s2.mvms == s1.mvms
        if prec == "mixed":
            _, xd = solve(pp, h, f, b, "dw", pp.PP_ORTH_DCGS2)
            assert rel(x2, xs) <= max(3 * rel(xd, xs), 1e-12)
            assert s2.switch_iter == s1.switch_iter
        else:
            assert rel(x2, x1) < 1e-12
            assert rel(x2, xs) < 1e-10
    finally:
        pp.pp_destroy(h)


def test_dcgs2_mixed_switch_mid_run():
    # the precision switch in the middle of the run: the result takes the leading
    # columns from the double-word basis and the rest, with the column that held
    # the candidate at the switch, from the FP32 basis
    pp = load()
    dims = (40, 36, 30)
    n = int(np.prod(dims))
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 8)
        b = synth.rhs(n, 9)
        s1, x1 = solve(pp, h, 1, b, "mixed", pp.PP_ORTH_CGS2, tol=1e-10, check_every=2)
        s2, x2 = solve(pp, h, 1, b, "mixed", pp.PP_ORTH_DCGS2, tol=1e-10, check_every=2)
        _, xd = solve(pp, h, 1, b, "dw", pp.PP_ORTH_DCGS2, tol=1e-13)
        assert 0 < s2.switch_iter < s2.iters and s2.switch_iter == s1.switch_iter
        assert rel(x2, xd) < 1e-9 and rel(x1, xd) < 1e-9
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw"])
def test_dcgs2_csr_and_laplacian(prec):
    # a Hermitian operator through Arnoldi (no Lanczos) and a CSR handle
    pp = load()
    dims = (37, 29)
    n = int(np.prod(dims))
    rp, col, val = synth.stencil_csr("laplace2d5", dims)
    keep = [dev(a) for a in (rp, col, val)]
    h = pp.pp_create_csr(n, *keep, is_hermitian=True)
    try:
        pp.pp_build_poly(h, 7, interval_ab=ops.laplace_interval(dims))
        b = synth.rhs(n, 5)
        st, x = solve(pp, h, -1, b, prec, pp.PP_ORTH_DCGS2)
        assert st.status == pp.PP_OK
        assert rel(x, exact.separable_fun(dims, b, -0.5)) < 1e-10
    finally:
        pp.pp_destroy(h)


def test_dcgs2_graph_laplacian_example3():
    # Example 3's problem class (singular, non-normal CSR, Ritz q), Example 3's check cadence
    pp = load()
    from tests.test_gpu_graph import N, graph, reference
    rp, col, val = graph()
    keep = [dev(a) for a in (rp, col, val)]
    h = pp.pp_create_csr(N, *keep, is_hermitian=False)
    try:
        for degree, kind in ((7, pp.PP_RITZ_LEJA), (15, pp.PP_HARMONIC_RITZ)):
            pp.pp_build_poly(h, degree, kind)
            b, xref = reference(4)
            st, x = solve(pp, h, pp.PP_SQRT, b, "dw", pp.PP_ORTH_DCGS2, tol=1e-11, m_max=800,
                          check_every=max(1, 32 // (degree + 1)))
            assert st.status == pp.PP_OK
            assert rel(x, xref) < 1e-7
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw"])
def test_dcgs2_lucky_breakdown(prec):
    # 60 unknowns: the Krylov space becomes invariant before m_max
    pp = load()
    dims = (5, 4, 3)
    n = int(np.prod(dims))
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 0)
        b = synth.rhs(n, 3)
        st, x = solve(pp, h, -1, b, prec, pp.PP_ORTH_DCGS2, tol=1e-15, m_max=200, check_every=1)
        assert st.status == pp.PP_OK and st.iters <= n
        assert rel(x, exact.separable_fun(dims, b, -0.5, "convdiff", 0.5)) < 1e-10
    finally:
        pp.pp_destroy(h)


def test_dcgs2_refusals():
    pp = load()
    dims = (9, 8, 7)
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 4)
        o = pp.pp_default_opts()
        o.orth = pp.PP_ORTH_DCGS2
        o.side = pp.PP_RIGHT
        pp.pp_set_opts(h, o)
        b = torch.zeros(504, dtype=torch.float64, device="cuda") + 1.0
        x = torch.empty_like(b)
        with pytest.raises(pp.PPError) as e:
            pp.pp_apply(h, -1, b, x)
        assert e.value.status == pp.PP_ERR_UNSUPPORTED
        o.orth = 4
        with pytest.raises(pp.PPError) as e:
            pp.pp_set_opts(h, o)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(h)
