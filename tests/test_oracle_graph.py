"""Pins of the in-degree graph Laplacian inputs and of the oracle on them
(Sec. 6, Example 3: L = D_in - A of a directed graph, L^{1/2} b through
L^{-1/2}(L b), Sec. 4 / Thm. 4.1).  CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import synth
from oracle import exact, krylov, ritz


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def graph(n, m, seed=5):
    src, dst = synth.directed_powerlaw_graph(n, m, seed=seed)
    rp, col, val = synth.graph_laplacian_csr(n, src, dst)
    return src, dst, sp.csr_matrix((val, col, rp), shape=(n, n))


def test_graph_generator_structure():
    n, m = 2000, 15000
    src, dst, L = graph(n, m)
    assert len(src) == m
    assert np.all(src != dst)
    assert len(np.unique(src * n + dst)) == m
    assert np.bincount(dst, minlength=n).min() >= 1       # every node has an in-link
    # L = D_in - A: off-diagonal -1 per edge i -> j at (i, j), columns sum to zero
    assert np.abs(np.asarray(L.sum(axis=0))).max() == 0.0
    assert L.nnz == m + n
    A = sp.csr_matrix((np.ones(m), (src, dst)), shape=(n, n))
    assert (sp.diags(np.asarray(A.sum(axis=0)).ravel()) - A - L).count_nonzero() == 0
    # power-law in-degrees: a few hubs hold a large share of the edges
    indeg = np.sort(np.bincount(dst, minlength=n))[::-1]
    assert indeg[:20].sum() > 0.2 * m


def test_laplacian_spectrum_right_half_plane_semisimple_zero():
    # Gershgorin on the columns: spec(L) in the closed right half-plane; the
    # zero eigenvalue is semi-simple (rank L = rank L^2), as Thm. 4.1 needs
    n = 400
    _, _, L = graph(n, 2800, seed=9)
    Ld = L.toarray()
    lam = np.linalg.eigvals(Ld)
    assert lam.real.min() > -1e-9 * np.abs(lam).max()
    assert np.abs(lam).min() < 1e-9 * np.abs(lam).max()
    r1 = np.linalg.matrix_rank(Ld, tol=1e-8 * np.abs(lam).max())
    r2 = np.linalg.matrix_rank(Ld @ Ld, tol=1e-8 * np.abs(lam).max() ** 2)
    assert r1 == r2 < n


@pytest.mark.parametrize("seed", [4, 11])
def test_sqrt_of_singular_laplacian(seed):
    # L^{1/2} e_i by Algorithm 1 on L^{-1/2}(L e_i) (plain Arnoldi with CGS2)
    # against the principal square root of the dense matrix, and the identity
    # (L^{1/2})^2 e_i = L e_i
    n = 300
    _, _, L = graph(n, 2100, seed=9)
    Ld = L.toarray()
    b = synth.unit_vector(n, seed)
    ref = np.real(sla.sqrtm(Ld) @ b)
    r = krylov.pp_arnoldi(L.dot, b, 0.5, m_max=n, tol=1e-13, k_chk=4, orth="cgs2")
    assert r["converged"]
    # z^{1/2} is ill-conditioned next to the zero eigenvalue: the Schur
    # (sqrtm) and the eigendecomposition forms of the dense root already
    # differ by ~3e-9 here, so 2e-8 is the agreement to expect
    assert rel(r["x"], ref) < 2e-8
    r2 = krylov.pp_arnoldi(L.dot, r["x"], 0.5, m_max=n, tol=1e-13, k_chk=4, orth="cgs2")
    assert rel(r2["x"], L @ b) < 2e-8


@pytest.mark.parametrize("harmonic", [False, True])
def test_ritz_preconditioned_sqrt_of_laplacian(harmonic):
    # Example 3's method: Ritz (or harmonic Ritz) q of degree 7 from the
    # library's start vector, Arnoldi with reorthogonalization, against plain
    # Arnoldi at a strict tolerance (the paper's reference)
    n = 600
    _, _, L = graph(n, 4500, seed=9)
    b = synth.unit_vector(n, 4)
    x, a = ritz.ritz_poly(L.dot, n, 7, harmonic=harmonic, hermitian=False)
    assert np.all(np.real(x) > 0)
    r = krylov.pp_arnoldi(L.dot, b, 0.5, q=(7, lambda v: ritz.newton_apply(L.dot, a, x, v)), m_max=300,
                          tol=1e-11, k_chk=4, orth="cgs2")
    ref = krylov.pp_arnoldi(L.dot, b, 0.5, m_max=n, tol=1e-13, k_chk=4, orth="cgs2")
    assert r["converged"] and ref["converged"]
    assert rel(r["x"], ref["x"]) < 1e-9
    assert r["iters"] < ref["iters"]
