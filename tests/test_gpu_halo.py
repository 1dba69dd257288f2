"""Paired stencil steps through TMA-staged halo tiles (pp_opts.halo) on the GPU.

A pair of real-node Horner steps evaluated in one launch uses the expression
order of the single-step kernel, so a solve with opts.halo = 1 must return
the same iterate bit for bit as with opts.halo = 0, with the same iteration
and operator counts and fewer launches whenever pairs ran.  The cases:
3D convection-diffusion and the 2D Laplacian on grids that end in partial
tiles, FP32 from the start (a loose tolerance) and after a precision switch,
both functions; grids that do not qualify (nx % 4 != 0) and q with conjugate
pairs run single steps (the same launches).  Against the FP64 oracle's closed
form the 2D Laplacian result keeps the mixed-precision bound of the other
tests.
"""
import numpy as np
import pytest

import synth
from oracle import exact
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solve(pp, h, f, b, halo, tol, prec=2, m_max=400):
    o = pp.pp_default_opts()
    o.precision = prec
    o.halo = halo
    pp.pp_set_opts(h, o)
    x = torch.empty(b.shape[0], dtype=torch.float64, device="cuda")
    st = pp.pp_apply(h, f, dev(b), x, m_max=m_max, tol=tol)
    torch.cuda.synchronize()
    return st, x.cpu().numpy()


CASES = [
    ("convdiff3d7", (36, 20, 13), [0.5], 16),   # partial tiles in y and z
    ("convdiff3d7", (64, 32, 16), [0.5], 9),    # whole tiles, odd degree (a single last step)
    ("laplace3d7", (20, 12, 6), None, 12),
    ("laplace2d5", (68, 40), None, 16),         # partial tiles in x and y
    ("laplace2d5", (256, 96), None, 7),
]


@pytest.mark.parametrize("f", [1, -1], ids=["sqrt", "invsqrt"])
@pytest.mark.parametrize("tol", [1e-5, 1e-10], ids=["fp32_from_start", "after_switch"])
@pytest.mark.parametrize("kind,dims,params,degree", CASES)
def test_pairs_bitwise_single_steps(kind, dims, params, degree, tol, f):
    pp = load()
    sk = {"convdiff3d7": pp.PP_CONVDIFF3D7_UPWIND, "laplace3d7": pp.PP_LAPLACE3D7,
          "laplace2d5": pp.PP_LAPLACE2D5}[kind]
    n = int(np.prod(dims))
    h = pp.pp_create_stencil(sk, dims, params)
    try:
        pp.pp_build_poly(h, degree)
        b = synth.rhs(n, 17)
        s0, x0 = solve(pp, h, f, b, 0, tol)
        s1, x1 = solve(pp, h, f, b, 1, tol)
        assert s0.status == s1.status == pp.PP_OK
        assert np.array_equal(x0, x1)
        assert (s1.iters, s1.mvms, s1.switch_iter) == (s0.iters, s0.mvms, s0.switch_iter)
        if s0.switch_iter == 0:
            assert s1.launches < s0.launches  # pairs ran from the first step on
        assert s1.launches <= s0.launches
        # a replay of the captured segment graphs gives the same again
        s2, x2 = solve(pp, h, f, b, 1, tol)
        assert np.array_equal(x1, x2) and s2.iters == s1.iters
    finally:
        pp.pp_destroy(h)


def test_pairs_against_closed_form_2d():
    pp = load()
    dims = (132, 72)
    n = dims[0] * dims[1]
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    try:
        pp.pp_build_poly(h, 16)
        b = synth.rhs(n, 3)
        st, x = solve(pp, h, -1, b, 1, 1e-10)
        assert st.status == pp.PP_OK and st.switch_iter >= 0
        xs = exact.separable_fun(dims, b, -0.5)
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    finally:
        pp.pp_destroy(h)


def test_unqualified_grids_and_conjugate_pairs_run_single_steps():
    pp = load()
    # nx % 4 != 0: the row pitch is not a multiple of 16 bytes
    dims = (30, 17, 9)
    n = int(np.prod(dims))
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 8)
        b = synth.rhs(n, 5)
        s0, x0 = solve(pp, h, 1, b, 0, 1e-6)
        s1, x1 = solve(pp, h, 1, b, 1, 1e-6)
        assert np.array_equal(x0, x1) and s0.launches == s1.launches
    finally:
        pp.pp_destroy(h)
    # Ritz q of a non-symmetric operator: complex conjugate node pairs
    # (steps that read the vector two steps back) keep the single steps
    dims = (32, 16, 8)
    n = int(np.prod(dims))
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [1.5])
    try:
        pp.pp_build_poly(h, 10, pp.PP_RITZ_LEJA)
        _, nodes, _ = pp.pp_get_poly_nodes(h)
        b = synth.rhs(n, 6)
        s0, x0 = solve(pp, h, 1, b, 0, 1e-6)
        s1, x1 = solve(pp, h, 1, b, 1, 1e-6)
        assert np.array_equal(x0, x1)
        if np.any(np.abs(np.imag(nodes)) > 0):
            assert s0.launches == s1.launches
    finally:
        pp.pp_destroy(h)


def test_halo_option_validated():
    pp = load()
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, (8, 8))
    try:
        o = pp.pp_default_opts()
        o.halo = 2
        with pytest.raises(pp.PPError) as e:
            pp.pp_set_opts(h, o)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(h)
