"""Pins of the oracle's multi-threaded CSR product (oracle/spmv.py) against
scipy's sparse product and a dense matrix-vector product (library routines)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import spmv


def _rand_csr(n, density, seed, cplx=False, empty_rows=()):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=rng, format="lil")
    if cplx:
        B = sp.random(n, n, density=density, random_state=rng, format="lil")
        A = A.astype(np.complex128) + 1j * B
        A = sp.lil_matrix(A)
    for r in empty_rows:
        A[r, :] = 0
    return sp.csr_matrix(A)


@pytest.mark.parametrize("cplx_a,cplx_x", [(False, False), (True, True), (False, True)])
def test_matches_scipy_and_dense(cplx_a, cplx_x):
    A = _rand_csr(301, 0.03, 1, cplx_a, empty_rows=(0, 7, 300))
    rng = np.random.default_rng(2)
    x = rng.standard_normal(301) + (1j * rng.standard_normal(301) if cplx_x else 0.0)
    y = spmv.CsrMv(A)(x)
    assert y.dtype == (np.complex128 if (cplx_a or cplx_x) else np.float64)
    np.testing.assert_allclose(y, A.dot(x), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(y, A.toarray() @ x, rtol=1e-12, atol=1e-12)
    assert y[0] == 0 and y[7] == 0 and y[300] == 0


def test_stencil_operator():
    from oracle import operators as ops
    A = ops.convdiff((9, 8, 7), 0.5)
    x = np.random.default_rng(3).standard_normal(A.shape[0])
    np.testing.assert_allclose(spmv.CsrMv(A)(x), A.dot(x), rtol=1e-14, atol=1e-14)


def test_kernel_is_built_and_threaded():
    spmv.build()
    assert spmv.threads() >= 1
    assert spmv._load() is not False
