"""Pins of the oracle's least-squares contour polynomial (Sec. 5.3).  CPU only."""
import numpy as np
import pytest

import synth
from oracle import exact, krylov, lsq, operators as ops


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def test_basis_is_orthonormal_arnoldi():
    z = lsq.contour(np.array([1 + 0.5j, 1 - 0.5j, 3.0, 4 + 1j, 4 - 1j, 6.0]), 0.5, 300)
    d = 12
    P, H = lsq.basis(z, d)
    assert np.abs(P.conj().T @ P - np.eye(d)).max() < 1e-12
    assert np.allclose(P[:, 0], 1 / np.sqrt(len(z)))
    assert np.abs(z[:, None] * P[:, :d - 1] - P @ H).max() < 1e-12
    # points symmetric about the real axis: the basis polynomials are real
    assert np.abs(H.imag).max() < 1e-12


def test_interpolation_when_points_equal_degree():
    # N = d points: the least-squares polynomial interpolates z^{-1/2}
    z = np.array([0.5, 1.0, 2.0 + 1.0j, 2.0 - 1.0j, 3.5])
    P, H = lsq.basis(z, len(z))
    a = lsq.coeffs(P, z ** -0.5)
    assert np.allclose(lsq.evaluate(H, a, len(z), z), z ** -0.5, rtol=1e-11)


def test_least_squares_matches_vandermonde_lstsq():
    z = lsq.contour(np.array([0.7 + 0.4j, 0.7 - 0.4j, 5.0]), 0.3, 200)
    d = 7
    P, H = lsq.basis(z, d)
    a = lsq.coeffs(P, z ** -0.5)
    V = np.vander(z, d, increasing=True)
    c, *_ = np.linalg.lstsq(V, z ** -0.5, rcond=None)
    w = np.array([0.9, 2.0 + 0.3j, 4.2])
    assert np.allclose(lsq.evaluate(H, a, len(z), w), np.polynomial.polynomial.polyval(w, c), rtol=1e-8)
    # q is real on the real axis (symmetric points, f(conj z) = conj f(z))
    x = np.linspace(0.5, 5, 11)
    assert np.abs(lsq.evaluate(H, a, len(z), x).imag).max() < 1e-12


def test_maximum_modulus_inside_contour():
    # z^{-1/2} - q is holomorphic inside a contour that excludes (-inf, 0]:
    # its modulus inside is bounded by its maximum on the contour (Sec. 5.3);
    # a fine discretization stands in for the contour
    th = np.array([1 + 0.5j, 1 - 0.5j, 3.0, 4 + 1j, 4 - 1j, 6.0])
    z = lsq.contour(th, 0.5, 2000)
    P, H = lsq.basis(z, 10)
    a = lsq.coeffs(P, z ** -0.5)
    on = np.abs(z ** -0.5 - lsq.evaluate(H, a, len(z), z)).max()
    inside = np.array([2.0, 3.0 + 0.3j, 4.0 - 0.5j, 1.2 + 0.1j, 5.0])
    err_in = np.abs(inside ** -0.5 - lsq.evaluate(H, a, len(z), inside))
    assert err_in.max() <= on * (1 + 1e-9)


def test_apply_matches_evaluate_on_diagonal_and_eigen_form():
    z = lsq.contour(np.array([0.8 + 0.6j, 0.8 - 0.6j, 7.5]), 0.4, 400)
    P, H = lsq.basis(z, 9)
    a = lsq.coeffs(P, z ** -0.5)
    dg = np.linspace(0.8, 7.0, 50)
    assert np.allclose(lsq.apply(lambda u: dg * u, H, a, len(z), np.ones(50)),
                       lsq.evaluate(H, a, len(z), dg).real, rtol=1e-10)
    A = ops.laplace((7, 6)).toarray()
    lam, Q = np.linalg.eigh(A)
    v = synth.rhs(42, 3)
    want = Q @ (lsq.evaluate(H, a, len(z), lam).real * (Q.T @ v))
    assert rel(lsq.apply(lambda u: A @ u, H, a, len(z), v), want) < 1e-10


def test_contour_construction():
    th = np.array([1 + 0.5j, 1 - 0.5j, 3.0, 4 + 1j, 4 - 1j, 6.0, 0.2 + 0.3j, 0.2 - 0.3j])
    z = lsq.contour(th, 0.5, 400)
    assert len(z) == 398
    # symmetric about the real axis, nothing inside |z| < r_min (to the
    # chord error of the dense resampling), the hull's extent
    assert np.allclose(np.sort_complex(z), np.sort_complex(z.conj()))
    assert np.abs(z).min() > 0.5 * (1 - 1e-4)
    assert np.isclose(z.real.max(), 6.0) and np.isclose(z.imag.max(), 1.0, atol=0.02)
    # all-real Ritz values: the segment from max(min, r_min) to max
    s = lsq.contour(np.array([0.05, 2.0, 9.0]), 0.1, 50)
    assert np.isclose(s.real.min(), 0.1) and np.isclose(s.real.max(), 9.0) and np.all(s.imag == 0)


@pytest.mark.parametrize("power", [-0.5, 0.5])
def test_lsq_preconditioned_solve(power):
    # convection-diffusion: contour from Ritz values of the spectrum's hull
    # (here the exact real interval, made into a thin symmetric contour)
    dims = (7, 6, 5)
    A = ops.convdiff(dims, 0.5)
    a, b = ops.convdiff_interval(dims, 0.5)
    th = np.array([a, b, 0.5 * (a + b) + 0.3j, 0.5 * (a + b) - 0.3j])
    z = lsq.contour(th, 0.5 * a, 600)
    deg = 6
    P, H = lsq.basis(z, deg + 1)
    al = lsq.coeffs(P, z ** -0.5)
    assert lsq.evaluate(H, al, len(z), z).real.min() > 0  # q in C+ on the contour
    rhs = synth.rhs(A.shape[0], 2)
    r = krylov.pp_arnoldi(A.dot, rhs, power, q=(deg, lambda v: lsq.apply(A.dot, H, al, len(z), v)), m_max=200,
                          tol=1e-12, k_chk=2, orth="cgs2")
    assert r["converged"]
    assert rel(r["x"], exact.dense_fun(A.toarray(), rhs, power, hermitian=False)) < 1e-10
