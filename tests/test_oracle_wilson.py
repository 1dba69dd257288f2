"""Pins of the oracle's Wilson-type operator (oracle/wilson.py) against what
the mathematics fixes: the Clifford algebra of the gamma matrices, the
free-field Fourier closed form of A = D^H D, gamma_5-hermiticity of D, and
gauge covariance of D and of f(A).  The input generator of the links (Haar
SU(3)) is checked for unitarity and unit determinant."""
import numpy as np
import pytest

import synth
from oracle import exact, krylov, wilson


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def test_gamma_algebra():
    g = wilson.gammas()
    I4 = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2.0 * I4 * (mu == nu))
        assert np.allclose(g[4] @ g[mu] + g[mu] @ g[4], 0)
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))


def test_haar_links_are_su3():
    U = synth.wilson_links((2, 3, 2, 2), seed=1).astype(np.complex128).reshape(-1, 3, 3)
    eye = np.broadcast_to(np.eye(3), U.shape)
    assert np.allclose(U @ np.conj(np.transpose(U, (0, 2, 1))), eye, atol=1e-6)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-6)
    # left invariance in distribution is not testable cheaply; the mean of U vanishes for Haar
    big = synth.haar_su3(20000, np.random.default_rng(0))
    assert np.abs(big.mean(axis=0)).max() < 0.02


@pytest.mark.parametrize("dims", [(4, 3, 2, 6), (2, 2, 2, 4)])
def test_free_field_closed_form(dims):
    # P8: U = 1, A b from the sparse matrix equals the Fourier multiplier
    m0 = 0.1
    A = wilson.dhd_matrix(dims, synth.unit_links(dims), m0)
    b = synth.spinor_field(dims, 0)
    assert rel(A @ b, wilson.free_field_fun(dims, b, 1.0, m0)) < 1e-13
    # and the closed-form spectrum with multiplicity 12
    if A.shape[0] <= 600:
        lam = np.sort(np.linalg.eigvalsh(A.toarray()))
        ref = np.sort(np.repeat(wilson.free_eigs(dims, m0).reshape(-1), 12))
        assert np.allclose(lam, ref, rtol=0, atol=1e-12)


def test_free_field_inverse_sqrt_dense():
    dims = (2, 3, 2, 4)
    m0 = 0.1
    A = wilson.dhd_matrix(dims, synth.unit_links(dims), m0)
    b = synth.spinor_field(dims, 1)
    # kappa(A) = (m0 + 8)^2 / m0^2 = 6561: the dense eigendecomposition's
    # rounding is about kappa * u = 1.5e-12
    for power in (-0.5, 0.5):
        xd = exact.dense_fun(A, b, power, hermitian=True)
        assert rel(wilson.free_field_fun(dims, b, power, m0), xd) < 1e-11


def test_gamma5_hermiticity():
    dims = (3, 2, 2, 4)
    D = wilson.dirac_matrix(dims, synth.wilson_links(dims, 1), 0.1)
    b = synth.spinor_field(dims, 2)
    # D^H b = gamma5 D gamma5 b
    lhs = D.conj().T @ b
    rhs = wilson.gamma5_apply(D @ wilson.gamma5_apply(b))
    assert rel(lhs, rhs) < 1e-14


def test_gauge_covariance():
    dims = (2, 2, 3, 2)
    m0 = 0.1
    U = synth.wilson_links(dims, 1)
    G = synth.haar_su3(int(np.prod(dims)), np.random.default_rng(7))
    Ug = wilson.gauge_transform(dims, U, G)
    b = synth.spinor_field(dims, 3)
    D = wilson.dirac_matrix(dims, U, m0)
    Dg = wilson.dirac_matrix(dims, Ug, m0)
    assert rel(Dg @ wilson.gauge_apply(G, b), wilson.gauge_apply(G, D @ b)) < 1e-13
    A = wilson.dhd_matrix(dims, U, m0)
    Ag = wilson.dhd_matrix(dims, Ug, m0)
    x = exact.dense_fun(A, b, -0.5, hermitian=True)
    xg = exact.dense_fun(Ag, wilson.gauge_apply(G, b), -0.5, hermitian=True)
    assert rel(xg, wilson.gauge_apply(G, x)) < 1e-12


def test_lanczos_reference_matches_dense():
    # the large-lattice reference (plain Lanczos/Arnoldi, tight tolerance) on a random field
    dims = (2, 3, 2, 4)
    m0 = 0.1
    A = wilson.dhd_matrix(dims, synth.wilson_links(dims, 1), m0)
    b = synth.spinor_field(dims, 4)
    xd = exact.dense_fun(A, b, -0.5, hermitian=True)
    r = krylov.plain_reference(A.dot, b, -0.5, tol=1e-13, m_max=400, k_chk=4, hermitian=True)
    assert rel(r["x"], xd) < 1e-11


def test_mutation_is_caught():
    # planted mistake: the projectors of the two hops swapped (that is D^H, not
    # D, for the free field a different operator only through the sign of the
    # sin terms, so the free-field spectrum cannot see it) -- gamma5-hermiticity
    # of the planted operator against the true D fails on a random field
    dims = (2, 2, 2, 2)
    U = synth.wilson_links(dims, 1)
    D = wilson.dirac_matrix(dims, U, 0.1)
    g = wilson.gammas()
    saved = wilson.gammas
    try:
        wilson.gammas = lambda: [-m for m in g[:4]] + [g[4]]
        Dbad = wilson.dirac_matrix(dims, U, 0.1)
    finally:
        wilson.gammas = saved
    b = synth.spinor_field(dims, 5)
    assert rel(Dbad @ b, D @ b) > 1e-3
    # the planted operator equals D^H: the test of hermiticity above is what separates them
    assert rel(Dbad @ b, D.conj().T @ b) < 1e-13
