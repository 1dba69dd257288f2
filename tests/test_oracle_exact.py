"""Pins of the oracle's exact solutions and operators (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import exact, operators as ops


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


@pytest.mark.parametrize("dims", [(8, 8), (16, 16), (6, 7, 5)])
@pytest.mark.parametrize("power", [-0.5, 0.5])
def test_closed_form_equals_dense(dims, power):
    # P1: sine-basis closed form vs dense eigendecomposition
    A = ops.laplace(dims)
    b = synth.rhs(A.shape[0], 0)
    assert rel(exact.separable_fun(dims, b, power), exact.dense_fun(A, b, power)) < 1e-13


@pytest.mark.parametrize("N", [6, 8])
@pytest.mark.parametrize("power", [-0.5, 0.5])
def test_convdiff_closed_form_equals_schur(N, power):
    # P7: diagonal-similarity closed form vs the Schur square root of the dense matrix
    dims = (N, N, N)
    A = ops.convdiff(dims, 0.5)
    b = synth.rhs(A.shape[0], 1)
    x1 = exact.separable_fun(dims, b, power, "convdiff", 0.5)
    x2 = exact.dense_fun(A, b, power, hermitian=False)
    assert rel(x1, x2) < 1e-12


def test_eigenvalues_closed_form():
    for dims in [(5, 7), (4, 3, 5)]:
        lam = np.sort(np.linalg.eigvalsh(ops.laplace(dims).toarray()))
        assert np.allclose(lam, np.sort(exact.separable_eigs(dims)), atol=1e-12)
        lo, hi = ops.laplace_interval(dims)
        assert abs(lo - lam[0]) < 1e-12 and abs(hi - lam[-1]) < 1e-12
    A = ops.convdiff((4, 5, 3), 0.5).toarray()
    lam = np.sort(np.linalg.eigvals(A).real)
    assert np.allclose(lam, np.sort(exact.separable_eigs((4, 5, 3), "convdiff", 0.5)), atol=1e-10)
    # Example 1's interval formula for the 3D Laplacian
    N = 9
    lo, hi = ops.laplace_interval((N, N, N))
    assert abs(lo - 6 * (1 - np.cos(np.pi / (N + 1)))) < 1e-14
    assert abs(hi - (12 - 6 * (1 - np.cos(np.pi / (N + 1))))) < 1e-13


@pytest.mark.parametrize("kind,dims,ch", [("laplace2d5", (7, 5), 0.0), ("laplace3d7", (4, 5, 6), 0.0),
                                          ("convdiff3d7", (4, 5, 6), 0.5)])
def test_synth_csr_matches_kron_sum(kind, dims, ch):
    rp, col, val = synth.stencil_csr(kind, dims, ch)
    n = int(np.prod(dims))
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    B = ops.laplace(dims) if kind.startswith("laplace") else ops.convdiff(dims, ch)
    assert abs(M - B).max() == 0.0
    assert np.all(np.diff(rp) > 0) and rp[-1] == val.shape[0]


def test_identities_dense():
    # P4 on the definitions: (A^{1/2})^2 b = A b and A^{-1/2} A^{1/2} b = b
    A = ops.convdiff((5, 4, 6), 0.5)
    b = synth.rhs(A.shape[0], 3)
    s = exact.dense_fun(A, b, 0.5, hermitian=False)
    assert rel(exact.dense_fun(A, s, 0.5, hermitian=False), A @ b) < 1e-12
    assert rel(exact.dense_fun(A, s, -0.5, hermitian=False), b) < 1e-12


def test_diagonal():
    # P5: diagonal A
    rng = np.random.default_rng(5)
    a = rng.uniform(0.5, 3.0, 40)
    b = synth.rhs(40, 0)
    for p in (-0.5, 0.5):
        assert rel(exact.dense_fun(np.diag(a), b, p), exact.diagonal_fun(a, b, p)) < 1e-14
        assert np.allclose(exact.diagonal_fun(a, b, p), a ** p * b, rtol=1e-15)
