"""pp_poly_apply_static: q(A) x with no device allocation.

Some callers cannot let this library call cudaMalloc: a process whose GPU
memory is already owned by a framework's arena or caching allocator, or a
latency-critical loop that forbids allocation (and the device
synchronisation cudaFree implies) after start-up.  pp_poly_apply_static
serves them by taking its scratch vectors from one fixed array compiled into
the library instead of the handle's workspace.

These tests call it through the C ABI and check that it returns what
pp_poly_apply returns, within the q(A) v tolerance of the parity tests
(relative 2-norm 1e-12 in FP64, 5e-12 in double-word, 1e-7 (deg + 1) in the
FP32 arithmetic of PP_PREC_MIXED), on two calls in a row with different
inputs (the array is shared by every call and keeps the previous call's
contents).  A fresh handle whose first call is the static one is compared
with pp_poly_apply on a second handle, and the free device memory is checked
to stay the same across static calls.  They also check that sizes above the
array's capacity are refused.  The file is named so that pytest collects it
last.
"""
import numpy as np
import pytest

import synth
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 5e-12}  # pp_opts.precision -> tolerance (FP32: tol_f32(degree))


def tol_f32(degree):
    return 1e-7 * (degree + 1)


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def run_pair(pp, h, n, seeds):
    """q(A) b for each seed by both entry points; returns relative differences."""
    out = []
    for seed in seeds:
        b = torch.from_numpy(synth.rhs(n, seed)).cuda()
        y_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        y_static = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        pp.pp_poly_apply(h, b, y_ref)
        pp.pp_poly_apply_static(h, b, y_static)
        torch.cuda.synchronize()
        out.append(rel(y_static.cpu().numpy(), y_ref.cpu().numpy()))
    return out


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "dw", "mixed"])
@pytest.mark.parametrize("kind,dims,params,degree", [
    ("convdiff3d7", (33, 17, 29), [0.5], 9),
    ("laplace2d5", (61, 37), None, 16),
    ("laplace3d7", (64, 64, 64), None, 5),  # n = PP_STATIC_MAX_N exactly
    ("laplace2d5", (7, 5), None, 0),        # degree 0: q is a constant
])
def test_static_matches_workspace_version(kind, dims, params, degree, prec):
    pp = load()
    sk = {"convdiff3d7": pp.PP_CONVDIFF3D7_UPWIND, "laplace2d5": pp.PP_LAPLACE2D5,
          "laplace3d7": pp.PP_LAPLACE3D7}[kind]
    stream = torch.cuda.current_stream()
    h = pp.pp_create_stencil(sk, dims, params, stream=stream)
    try:
        o = pp.pp_default_opts()
        o.precision = prec
        pp.pp_set_opts(h, o)
        pp.pp_build_poly(h, degree)
        n = int(np.prod(dims))
        assert n <= pp.PP_STATIC_MAX_N
        diffs = run_pair(pp, h, n, seeds=(11, 12))
        tol = TOL[prec] if prec in TOL else tol_f32(degree)
        assert all(d <= tol for d in diffs), diffs
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "dw", "mixed"])
def test_static_first_on_fresh_handle_allocates_nothing(prec):
    # the static call is the handle's first device work (no workspace exists);
    # the result equals pp_poly_apply's on a second handle of the same operator
    pp = load()
    dims, degree = (45, 31, 17), 12
    n = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    hs = [pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5], stream=stream) for _ in range(2)]
    try:
        for h in hs:
            o = pp.pp_default_opts()
            o.precision = prec
            pp.pp_set_opts(h, o)
            pp.pp_build_poly(h, degree)
        bs = [torch.from_numpy(synth.rhs(n, s)).cuda() for s in (31, 32)]
        ys = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in bs]
        torch.cuda.synchronize()
        pp.pp_poly_apply_static(hs[0], bs[0], ys[0])  # first call: looks the array up on this device
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pp.pp_poly_apply_static(hs[0], bs[1], ys[1])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0  # no device allocation by the static call
        tol = TOL[prec] if prec in TOL else tol_f32(degree)
        # the oracle's q(A) v: the same Chebyshev interpolant by its three-term recurrence
        from oracle import chebyshev as cheb, operators as ops
        A = ops.convdiff(dims, 0.5)
        a, b_ = ops.convdiff_interval(dims, 0.5)
        c = cheb.interp_coeffs(a, b_, degree + 1)
        for b, y in zip(bs, ys):
            y_ref = torch.empty_like(b)
            pp.pp_poly_apply(hs[1], b, y_ref)
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            assert rel(yh, y_ref.cpu().numpy()) <= tol
            assert rel(yh, cheb.q_apply(A.dot, c, a, b_, b.cpu().numpy())) <= tol
    finally:
        for h in hs:
            pp.pp_destroy(h)


def test_static_csr_f64_and_refusals():
    pp = load()
    dims = (19, 23, 9)
    n = int(np.prod(dims))
    rp, col, val = synth.stencil_csr("convdiff3d7", dims, 0.5)
    keep = [torch.from_numpy(a).cuda() for a in (rp, col, val)]
    h = pp.pp_create_csr(n, *keep, is_hermitian=False, stream=torch.cuda.current_stream())
    try:
        pp.pp_build_poly(h, 7, interval_ab=(0.3, 17.5))
        diffs = run_pair(pp, h, n, seeds=(21, 22))
        assert all(d <= TOL[0] for d in diffs), diffs
        # double-word CSR would need a converted copy of the values: refused
        o = pp.pp_default_opts()
        o.precision = pp.PP_PREC_DW
        pp.pp_set_opts(h, o)
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(b)
        with pytest.raises(pp.PPError) as e:
            pp.pp_poly_apply_static(h, b, y)
        assert e.value.status == pp.PP_ERR_UNSUPPORTED
    finally:
        pp.pp_destroy(h)

    # one entry more than the array holds: refused before any device work
    big = pp.PP_STATIC_MAX_N + 1
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, (big, 1), stream=torch.cuda.current_stream())
    try:
        pp.pp_build_poly(h, 3)
        b = torch.zeros(big, dtype=torch.float64, device="cuda")
        y = torch.empty_like(b)
        with pytest.raises(pp.PPError) as e:
            pp.pp_poly_apply_static(h, b, y)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        assert "PP_STATIC_MAX_N" in pp.pp_last_error()
    finally:
        pp.pp_destroy(h)
