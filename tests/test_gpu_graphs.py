"""Segment graphs of pp_apply: the Krylov steps between two stopping checks
are captured once as a CUDA graph and replayed by later solves.  A replay
must give bitwise the result of direct launches (the same kernels with the
same arguments: opts.profile = 1 runs them directly), the same counters,
and a change of q, tolerance or options must not replay a stale graph."""
import numpy as np
import pytest

import synth
from oracle import exact, operators as ops
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def solve(pp, h, f, b, n, tol, profile, prec, dtype=torch.float64, orth=0):
    o = pp.pp_default_opts()
    o.precision = prec
    o.profile = profile
    o.orth = orth
    pp.pp_set_opts(h, o)
    x = torch.empty(n, dtype=dtype, device="cuda")
    st = pp.pp_apply(h, f, b, x, m_max=400, tol=tol)
    return host(x), st


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "dw", "mixed"])
@pytest.mark.parametrize("kind", ["laplace2d", "convdiff3d", "csr"])
def test_replay_is_bitwise_direct(kind, prec):
    pp = load()
    keep = []
    if kind == "laplace2d":
        dims = (61, 47)
        h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
        n, f = dims[0] * dims[1], -1
    elif kind == "convdiff3d":
        dims = (19, 17, 13)
        h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
        n, f = int(np.prod(dims)), 1
    else:
        dims = (40, 37)
        rp, col, val = synth.stencil_csr("laplace2d5", dims)
        keep = [dev(a) for a in (rp, col, val)]
        n, f = dims[0] * dims[1], -1
        h = pp.pp_create_csr(n, *keep, is_hermitian=True)
    try:
        pp.pp_build_poly(h, 8) if kind != "csr" else pp.pp_build_poly(h, 8, interval_ab=(0.005, 8.0))
        b = dev(synth.rhs(n, 3))
        x_direct, s0 = solve(pp, h, f, b, n, 1e-10, 1, prec)
        x_cap, s1 = solve(pp, h, f, b, n, 1e-10, 0, prec)      # captures
        x_rep, s2 = solve(pp, h, f, b, n, 1e-10, 0, prec)      # replays
        assert s0.status == s1.status == s2.status == pp.PP_OK
        assert np.array_equal(x_direct, x_cap) and np.array_equal(x_direct, x_rep)
        for st in (s1, s2):
            assert (st.iters, st.mvms, st.inner_products, st.switch_iter) == \
                (s0.iters, s0.mvms, s0.inner_products, s0.switch_iter)
            assert st.launches == s0.launches
        # another right-hand side through the same graphs
        b2 = dev(synth.rhs(n, 4))
        x2_direct, _ = solve(pp, h, f, b2, n, 1e-10, 1, prec)
        x2_rep, _ = solve(pp, h, f, b2, n, 1e-10, 0, prec)
        assert np.array_equal(x2_direct, x2_rep)
    finally:
        pp.pp_destroy(h)


def test_changes_invalidate_graphs():
    # tolerance, q and options change between solves: each result still
    # matches the exact solution (a stale graph would run the old q or tol)
    pp = load()
    dims = (33, 29)
    A = ops.laplace(dims)
    n = A.shape[0]
    b = synth.rhs(n, 0)
    xs = exact.dense_fun(A.toarray(), b, -0.5, hermitian=True)
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    try:
        bd = dev(b)
        for degree, tol, prec in [(4, 1e-6, 0), (4, 1e-11, 0), (12, 1e-11, 0), (12, 1e-11, 1), (0, 1e-11, 1)]:
            pp.pp_build_poly(h, degree)
            for _ in range(2):
                x, st = solve(pp, h, -1, bd, n, tol, 0, prec)
                assert st.status == pp.PP_OK
                assert rel(x, xs) < max(30 * tol, 1e-10)
    finally:
        pp.pp_destroy(h)


def test_complex_sign_replay():
    pp = load()
    dims = (2, 2, 2, 4)
    links = dev(synth.wilson_links(dims, 1).astype(np.complex64))
    h = pp.pp_create_stencil(pp.PP_WILSON4D_Q2, dims, [-1.4, 0.3], links=links, dtype=pp.PP_C128)
    n = 12 * int(np.prod(dims))
    try:
        pp.pp_build_poly(h, 4, pp.PP_RITZ_LEJA)
        b = dev(synth.spinor_field(dims, 0))
        xd, s0 = solve(pp, h, pp.PP_SIGN, b, n, 1e-12, 1, 1, torch.complex128)
        xc, s1 = solve(pp, h, pp.PP_SIGN, b, n, 1e-12, 0, 1, torch.complex128)
        xr, s2 = solve(pp, h, pp.PP_SIGN, b, n, 1e-12, 0, 1, torch.complex128)
        assert np.array_equal(xd, xc) and np.array_equal(xd, xr)
        assert s0.iters == s2.iters and s0.launches == s2.launches
    finally:
        pp.pp_destroy(h)


def test_multi_rhs_csr_and_wilson_columns():
    # nrhs > 1 on CSR and Wilson handles: the columns one after another, each
    # bitwise the single-column solve
    pp = load()
    dims = (30, 23)
    rp, col, val = synth.stencil_csr("laplace2d5", dims)
    keep = [dev(a) for a in (rp, col, val)]
    n = dims[0] * dims[1]
    h = pp.pp_create_csr(n, *keep, is_hermitian=True)
    try:
        pp.pp_build_poly(h, 6, interval_ab=(0.01, 8.0))
        B = np.stack([synth.rhs(n, s) for s in (1, 2, 3)], axis=1)
        X = torch.empty((3, n), dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, -1, dev(B.T.copy()), X, m_max=300, tol=1e-11, nrhs=3)
        assert st.status == pp.PP_OK
        for k in range(3):
            xk = torch.empty(n, dtype=torch.float64, device="cuda")
            s1 = pp.pp_apply(h, -1, dev(B[:, k].copy()), xk, m_max=300, tol=1e-11)
            assert np.array_equal(host(X[k]), host(xk))
            assert s1.iters <= st.iters
    finally:
        pp.pp_destroy(h)
    ldims = (2, 2, 2, 4)
    links = dev(synth.wilson_links(ldims, 1).astype(np.complex64))
    hq = pp.pp_create_stencil(pp.PP_WILSON4D_Q2, ldims, [-1.4, 0.3], links=links, dtype=pp.PP_C128)
    nq = 12 * int(np.prod(ldims))
    try:
        pp.pp_build_poly(hq, 4, pp.PP_RITZ_LEJA)
        B = np.stack([synth.spinor_field(ldims, s) for s in (0, 5)], axis=0)
        X = torch.empty((2, nq), dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(hq, pp.PP_SIGN, dev(B), X, m_max=200, tol=1e-12, nrhs=2)
        assert st.status == pp.PP_OK
        for k in range(2):
            xk = torch.empty(nq, dtype=torch.complex128, device="cuda")
            pp.pp_apply(hq, pp.PP_SIGN, dev(B[k].copy()), xk, m_max=200, tol=1e-12)
            assert np.array_equal(host(X[k]), host(xk))
    finally:
        pp.pp_destroy(hq)
