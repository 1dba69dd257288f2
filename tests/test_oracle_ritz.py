"""Pins of the oracle's Ritz / harmonic Ritz polynomials of Sec. 5.2 (CPU only)."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import chebyshev as cheb, exact, krylov, operators as ops, ritz


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def test_splitmix64_published_values():
    # the first three outputs of SplitMix64 started from state 0, as published
    # with the generator's reference implementation
    assert ritz.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert ritz.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert ritz.splitmix64(0, 2) == 0x06C45D188009454F


def test_start_values_match_scalar_definition():
    v = ritz.start_values(300, ritz.LIBRARY_SEED)
    for i in (0, 1, 7, 123, 299):
        s = ritz.splitmix64(ritz.LIBRARY_SEED, i)
        assert v[i] == (s >> 11) * 2.0 ** -52 - 1.0
    assert v.min() >= -1.0 and v.max() < 1.0
    # uniform on [-1, 1): mean near 0, variance near 1/3
    w = ritz.start_values(100000)
    assert abs(w.mean()) < 0.01 and abs(w.var() - 1.0 / 3.0) < 0.01
    z = ritz.start_vector(5, complex_=True)
    r = ritz.start_values(10)
    assert np.array_equal(z.real, r[0::2]) and np.array_equal(z.imag, r[1::2])


def test_arnoldi_relation_and_tridiagonal():
    A = ops.laplace((9, 7))
    n = A.shape[0]
    d = 12
    H, V = ritz.arnoldi(A.dot, ritz.start_vector(n), d)
    assert H.shape == (d + 1, d)
    # V orthonormal and A V_d = V_{d+1} H
    assert np.abs(V @ V.T - np.eye(d + 1)).max() < 1e-13
    assert np.abs(A @ V[:d].T - V.T @ H).max() < 1e-12
    # Hermitian A: tridiagonal up to rounding
    assert np.abs(np.triu(H[:d, :d], 2)).max() < 1e-12


def test_ritz_values_exact_space():
    # d = n: the Krylov space is the whole space; Ritz values = eigenvalues
    lam = np.array([0.3, 0.9, 1.7, 2.0, 4.5, 8.0])
    A = np.diag(lam)
    H, _ = ritz.arnoldi(lambda v: A @ v, ritz.start_vector(6), 6)
    assert np.allclose(ritz.ritz_values(H), lam, rtol=1e-12)
    assert np.allclose(ritz.harmonic_ritz_values(H), lam, rtol=1e-10)


def test_ritz_one_step_is_rayleigh_quotient():
    A = ops.laplace((6, 5))
    v = ritz.start_vector(30)
    H, _ = ritz.arnoldi(A.dot, v, 1)
    assert np.isclose(ritz.ritz_values(H)[0], v @ (A @ v) / (v @ v), rtol=1e-14)


@pytest.mark.parametrize("d", [1, 3, 8, 15])
def test_harmonic_ritz_is_pencil(d):
    # harmonic Ritz values: theta with A u - theta u orthogonal to A K_d, u in K_d,
    # i.e. the pencil (V^T A^2 V, V^T A V), solved here by a generalized symmetric solver
    A = ops.laplace((11, 9)).toarray()
    n = A.shape[0]
    H, V = ritz.arnoldi(lambda v: A @ v, ritz.start_vector(n), d)
    Vd = V[:d].T
    AV = A @ Vd
    pencil = np.sort(sla.eigh(AV.T @ AV, Vd.T @ AV, eigvals_only=True))
    h = ritz.harmonic_ritz_values(H)
    assert np.allclose(h, pencil, rtol=1e-9)
    lam = np.linalg.eigvalsh(A)
    # Sec. 5.2: the inverses lie in the field of values of A^{-1}; for SPD A
    # harmonic Ritz values are >= lambda_min (bounded away from 0), and <= lambda_max
    assert h.min() >= lam[0] * (1 - 1e-10) and h.max() <= lam[-1] * (1 + 1e-10)
    r = ritz.ritz_values(H)
    assert r.min() >= lam[0] * (1 - 1e-10) and r.max() <= lam[-1] * (1 + 1e-10)
    # harmonic values sit above the standard ones, one by one (both interlace
    # the same way; for SPD A the harmonic Rayleigh quotient dominates)
    assert np.all(h >= r * (1 - 1e-10))


def test_leja_hand_example():
    # worked by hand: start at 4 (largest modulus); then 0.5 (|z-4| = 3.5 is
    # largest); then 2 (products 1.5, 3, 1.5 for 1, 2, 3.5); then 3.5 (2.25 vs 1.5)
    x = ritz.leja_order([0.5, 1.0, 2.0, 3.5, 4.0])
    assert list(x) == [4.0, 0.5, 2.0, 3.5, 1.0]


def test_leja_properties():
    rng = np.random.default_rng(3)
    pts = np.sort(rng.uniform(0.1, 5.0, 17))
    x = ritz.leja_order(pts)
    assert np.array_equal(np.sort(x), pts)
    assert x[0] == pts[-1]
    # greedy: every chosen node maximizes the product over the nodes still left
    for k in range(1, len(x)):
        left = x[k:]
        prods = [np.prod(np.abs(z - x[:k])) for z in left]
        assert np.prod(np.abs(x[k] - x[:k])) >= max(prods) * (1 - 1e-12)


def test_newton_interpolates():
    rng = np.random.default_rng(4)
    x = ritz.leja_order(np.sort(rng.uniform(0.2, 9.0, 10)))
    a = ritz.newton_coeffs(x)
    assert np.allclose(ritz.newton_eval(a, x, x), x ** -0.5, rtol=1e-12)
    # the unique interpolant of degree 9: compare with a Vandermonde solve
    z = np.linspace(0.2, 9.0, 57)
    p = np.polynomial.polynomial.polyfit(x, x ** -0.5, len(x) - 1)
    assert np.allclose(ritz.newton_eval(a, x, z), np.polynomial.polynomial.polyval(z, p), rtol=1e-8)
    # the polynomial does not depend on the node order
    y = x[::-1].copy()
    assert np.allclose(ritz.newton_eval(ritz.newton_coeffs(y), y, z), ritz.newton_eval(a, x, z), rtol=1e-9)


def test_newton_at_chebyshev_nodes_is_chebyshev_interpolant():
    a, b, deg = 0.05, 8.0, 14
    t = np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1)
    nodes = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(t)
    x = ritz.leja_order(np.sort(nodes))
    an = ritz.newton_coeffs(x)
    c = cheb.interp_coeffs(a, b, deg + 1)  # d = deg + 1 nodes
    z = np.linspace(a, b, 301)
    assert np.allclose(ritz.newton_eval(an, x, z), cheb.q_eval(c, a, b, z), rtol=1e-10)


def test_newton_coeffs_of_a_polynomial():
    # divided differences of a cubic: a_3 = leading coefficient, a_k = 0 beyond
    x = np.array([3.0, 0.5, 1.5, 2.5, 1.0])
    a = ritz.newton_coeffs(x, f=lambda z: 2 * z ** 3 - z + 4)
    assert np.isclose(a[3], 2.0) and abs(a[4]) < 1e-12
    assert np.isclose(a[0], 2 * 27 - 3 + 4)


def test_newton_apply_matches_eigen_form():
    A = ops.laplace((8, 6)).toarray()
    lam, Q = np.linalg.eigh(A)
    x = ritz.leja_order(np.sort(np.linspace(0.3, 7.5, 9)))
    a = ritz.newton_coeffs(x)
    v = synth.rhs(A.shape[0], 1)
    got = ritz.newton_apply(lambda u: A @ u, a, x, v)
    want = Q @ (ritz.newton_eval(a, x, lam) * (Q.T @ v))
    assert rel(got, want) < 1e-12
    # diagonal matrix: entrywise
    dg = np.linspace(0.5, 6.0, 40)
    assert np.allclose(ritz.newton_apply(lambda u: dg * u, a, x, np.ones(40)), ritz.newton_eval(a, x, dg),
                       rtol=1e-12)


@pytest.mark.parametrize("harmonic", [False, True])
@pytest.mark.parametrize("power", [-0.5, 0.5])
def test_ritz_preconditioned_solve_converges(harmonic, power):
    dims = (30, 26)
    A = ops.laplace(dims)
    n = A.shape[0]
    b = synth.rhs(n, 5)
    deg = 7
    x, an = ritz.ritz_poly(A.dot, n, deg, harmonic=harmonic)
    assert len(x) == deg + 1
    # q interpolates z^{-1/2} at the nodes and is positive on the spectrum
    assert np.allclose(ritz.newton_eval(an, x, x), x ** -0.5, rtol=1e-10)
    lam = exact.separable_eigs(dims)
    assert ritz.newton_eval(an, x, lam).min() > 0
    r = krylov.pp_arnoldi(A.dot, b, power, q=(deg, lambda v: ritz.newton_apply(A.dot, an, x, v)),
                          m_max=120, tol=1e-12, k_chk=2, hermitian=True, orth="lanczos")
    assert r["converged"]
    assert rel(r["x"], exact.separable_fun(dims, b, power)) < 1e-10
    # preconditioning pays: fewer iterations than plain Lanczos
    r0 = krylov.pp_arnoldi(A.dot, b, power, m_max=400, tol=1e-12, k_chk=2, hermitian=True, orth="lanczos")
    assert r["iters"] < r0["iters"] / 2


def test_invariant_subspace_stops_early():
    A = np.diag([1.0, 2.0, 3.0])
    v = np.array([1.0, 1.0, 0.0])
    H, V = ritz.arnoldi(lambda u: A @ u, v, 3)
    assert H.shape == (3, 2)
    assert np.allclose(ritz.ritz_values(H), [1.0, 2.0])


# ---- non-Hermitian A: complex Ritz values in conjugate pairs ----

def same_set(a, b, tol):
    """Every entry of a within tol of an entry of b and vice versa (equal multisets up to rounding)."""
    a, b = np.asarray(a), np.asarray(b)
    return len(a) == len(b) and max(np.abs(b - z).min() for z in a) < tol and \
        max(np.abs(a - z).min() for z in b) < tol


def _nonnormal(n=40, seed=7):
    # real non-symmetric matrix with eigenvalues in the right half-plane, some
    # complex: a shifted upper triangle plus a random rotation block structure
    rng = np.random.default_rng(seed)
    A = np.diag(np.linspace(1.0, 6.0, n)) + 0.6 * np.triu(rng.standard_normal((n, n)), 1)
    for k in range(0, n - 1, 5):  # 2x2 rotation blocks give complex pairs
        A[k + 1, k] = -1.5
        A[k, k + 1] = 1.5
    return A


def test_leja_complex_pairs_adjacent():
    z = np.array([1.0, 2 + 1j, 2 - 1j, 4.0, 3 + 0.5j, 3 - 0.5j, 0.5])
    x = ritz.leja_order(z)
    assert len(x) == len(z) and np.allclose(np.sort_complex(x), np.sort_complex(z))
    assert x[0] == 4.0
    k = 0
    while k < len(x):
        if x[k].imag != 0:
            assert x[k].imag > 0 and x[k + 1] == x[k].conjugate()
            k += 2
        else:
            k += 1
    # worked by hand: after 4, the product |z - 4| is largest at 0.5 (3.5 vs
    # |2 +- i - 4| = 2.24, |3 +- 0.5i - 4| = 1.12, |1 - 4| = 3)
    assert x[1] == 0.5


def test_newton_complex_nodes_real_polynomial():
    x = ritz.leja_order(np.array([0.8, 1.5 + 0.7j, 1.5 - 0.7j, 3.0 + 1.2j, 3.0 - 1.2j, 5.0, 2.2]))
    a = ritz.newton_coeffs(x)
    # interpolation at every (complex) node, principal branch
    assert np.allclose(ritz.newton_eval(a, x, x), x ** -0.5, rtol=1e-12)
    # real on the real axis (conjugation-closed node set, f(conj z) = conj f(z))
    zr = np.linspace(0.5, 6.0, 101)
    qr = ritz.newton_eval(a, x, zr)
    assert np.abs(qr.imag).max() < 1e-13 * np.abs(qr).max()
    # the unique interpolant: a complex Vandermonde solve gives the same values
    V = np.vander(x, increasing=True)
    c = np.linalg.solve(V, x ** -0.5)
    assert np.allclose(np.polynomial.polynomial.polyval(zr, c), qr, rtol=1e-8)


def test_newton_apply_nonnormal_matches_eigen_form():
    A = _nonnormal(30, 3)
    lam, W = np.linalg.eig(A)
    x = ritz.leja_order(np.array([1.2, 2.0 + 1.0j, 2.0 - 1.0j, 4.5, 3.3]))
    a = ritz.newton_coeffs(x)
    v = synth.rhs(30, 2)
    got = ritz.newton_apply(lambda u: A @ u, a, x, v)
    assert not np.iscomplexobj(got)
    want = W @ (ritz.newton_eval(a, x, lam) * np.linalg.solve(W, v))
    assert np.abs(want.imag).max() < 1e-10 * np.abs(want).max()
    assert rel(got, want.real) < 1e-10


def test_nonhermitian_ritz_values_are_projection_eigenvalues():
    A = _nonnormal(40, 7)
    d = 9
    H, V = ritz.arnoldi(lambda u: A @ u, ritz.start_vector(40), d)
    Vd = V[:d].T
    proj = np.linalg.eigvals(Vd.T @ A @ Vd)
    th = ritz.ritz_values(H, hermitian=False)
    assert same_set(th, proj, 1e-10 * np.abs(proj).max())
    assert np.any(np.abs(th.imag) > 1e-3)  # the case exercises complex pairs
    # harmonic: A u - theta u orthogonal to A K_d, i.e. the pencil
    # ((A V)^T A V, (A V)^T V), solved by a generalized eigensolver
    AV = A @ Vd
    pen = sla.eigvals(AV.T @ AV, AV.T @ Vd)
    hh = ritz.harmonic_ritz_values(H, hermitian=False)
    assert same_set(hh, pen, 1e-8 * np.abs(pen).max())


@pytest.mark.parametrize("harmonic", [False, True])
def test_nonhermitian_ritz_solve(harmonic):
    # convection-diffusion (real, non-symmetric): q from the Arnoldi Ritz
    # values, Algorithm 1 with CGS2, against the dense definition
    dims = (7, 6, 5)
    A = ops.convdiff(dims, 0.5)
    n = A.shape[0]
    b = synth.rhs(n, 4)
    deg = 6
    x, an = ritz.ritz_poly(A.dot, n, deg, harmonic=harmonic, hermitian=False)
    assert len(x) == deg + 1
    q = (deg, lambda v: ritz.newton_apply(A.dot, an, x, v))
    for power in (-0.5, 0.5):
        r = krylov.pp_arnoldi(A.dot, b, power, q=q, m_max=200, tol=1e-12, k_chk=2, orth="cgs2")
        assert r["converged"]
        assert rel(r["x"], exact.dense_fun(A.toarray(), b, power, hermitian=False)) < 1e-10
