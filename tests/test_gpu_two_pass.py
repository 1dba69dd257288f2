"""Two-pass Lanczos (pp_opts.two_pass) through the C ABI.

Pass 2 regenerates the Lanczos vectors from the stored coefficients with the
same kernels, so the iterate equals the full-storage solve up to the order in
which x = V_m z is summed (column by column here): relative difference
1e-13.  Against the exact solution: 1e-10 (FP64 / double-word), mixed within
max(3 x the double-word error, tol) as for the full-storage solves.
"""
import numpy as np
import pytest

import synth
from oracle import exact
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def opts(pp, prec, side=0, two_pass=0, orth=0):
    o = pp.pp_default_opts()
    o.precision = prec
    o.side = side
    o.two_pass = two_pass
    o.orth = orth
    return o


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "dw", "mixed"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
@pytest.mark.parametrize("kind,dims,degree", [("laplace3d", (33, 17, 29), 8), ("laplace2d", (64, 38), 4)])
def test_two_pass_equals_full(kind, dims, degree, f, side, prec):
    pp = load()
    sk = pp.PP_LAPLACE3D7 if kind == "laplace3d" else pp.PP_LAPLACE2D5
    h = pp.pp_create_stencil(sk, dims)
    try:
        pp.pp_build_poly(h, degree)
        n = int(np.prod(dims))
        b = synth.rhs(n, 0)
        bd = torch.from_numpy(b).cuda()
        x1 = torch.empty(n, dtype=torch.float64, device="cuda")
        x2 = torch.empty_like(x1)
        pp.pp_set_opts(h, opts(pp, prec, side, 0))
        s1 = pp.pp_apply(h, f, bd, x1, m_max=400, tol=1e-11)
        pp.pp_set_opts(h, opts(pp, prec, side, 1))
        s2 = pp.pp_apply(h, f, bd, x2, m_max=400, tol=1e-11)
        torch.cuda.synchronize()
        assert s1.status == pp.PP_OK and s2.status == pp.PP_OK
        assert s2.iters == s1.iters and s2.switch_iter == s1.switch_iter
        X1, X2 = x1.cpu().numpy(), x2.cpu().numpy()
        assert rel(X2, X1) < 1e-13
        xs = exact.separable_fun(dims, b, 0.5 * f)
        if prec != 2:
            assert rel(X2, xs) < 1e-10
        else:
            pp.pp_set_opts(h, opts(pp, 1, side, 0))
            pp.pp_apply(h, f, bd, x1, m_max=400, tol=1e-11)
            torch.cuda.synchronize()
            assert rel(X2, xs) <= max(3 * rel(x1.cpu().numpy(), xs), 1e-11)
        # the second pass repeats the Krylov steps' operator work
        assert s2.mvms > s1.mvms
    finally:
        pp.pp_destroy(h)


def test_two_pass_full_size_laplace2048_mixed():
    # the 2048^2 Laplacian with O(n) basis memory, against the closed form
    pp = load()
    dims = (2048, 2048)
    n = dims[0] * dims[1]
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    try:
        pp.pp_build_poly(h, 16)
        pp.pp_set_opts(h, opts(pp, 2, 0, 1))
        b = synth.rhs(n, 0)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, -1, torch.from_numpy(b).cuda(), x, m_max=1000, tol=1e-9)
        torch.cuda.synchronize()
        assert st.status == pp.PP_OK
        assert rel(x.cpu().numpy(), exact.separable_fun(dims, b, -0.5)) < 1e-8
    finally:
        pp.pp_destroy(h)


def test_two_pass_needs_lanczos():
    pp = load()
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (10, 10, 10), [0.5])
    try:
        pp.pp_build_poly(h, 4)
        pp.pp_set_opts(h, opts(pp, 1, 0, 1))
        b = torch.from_numpy(synth.rhs(1000, 0)).cuda()
        x = torch.empty_like(b)
        with pytest.raises(pp.PPError) as e:
            pp.pp_apply(h, -1, b, x)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(h)
