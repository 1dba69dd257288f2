"""Pins of the oracle's Algorithms 1/2 (CPU only)."""
import os

import numpy as np
import pytest

import synth
from oracle import chebyshev as cheb, exact, krylov, operators as ops

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("orth", ["lanczos", "mgs", "cgs2"])
@pytest.mark.parametrize("power", [-0.5, 0.5])
def test_converges_to_closed_form(side, orth, power):
    dims = (32, 32)
    A = ops.laplace(dims)
    b = synth.rhs(A.shape[0], 0)
    a, bb = ops.laplace_interval(dims)
    c = cheb.interp_coeffs(a, bb, 9)
    # MGS loses orthogonality once the space is nearly invariant (the estimate then
    # stalls near 1e-12 for the A b start vector), so it gets a looser stopping tolerance
    tol = 1e-10 if orth == "mgs" else 1e-12
    r = krylov.pp_arnoldi(A.dot, b, power, c, (a, bb), side=side, m_max=200, tol=tol,
                          k_chk=7, hermitian=True, orth=orth)
    assert r["converged"]
    assert rel(r["x"], exact.separable_fun(dims, b, power)) < 1e-10
    deg = len(c) - 1
    # counters: 2d-1 mvms per iteration (Sec. 6, Example 1) plus the start-up products
    extra = (deg if side == "left" else 0) + (1 if power > 0 else 0)
    assert r["mvms"] == r["iters"] * (2 * deg + 1) + extra
    m = r["iters"]
    ip = {"lanczos": 2 * m, "mgs": m * (m + 1) // 2 + m, "cgs2": m * (m + 1) + m}[orth]
    assert r["inner_products"] == ip


def test_degree_zero_is_plain_arnoldi():
    # P4: a constant q only rescales A q^2; the Krylov space and the iterates are unchanged
    dims = (12, 10)
    A = ops.laplace(dims)
    b = synth.rhs(A.shape[0], 4)
    r1 = krylov.pp_arnoldi(A.dot, b, -0.5, (1.0,), side="left", m_max=25, tol=0.0, k_chk=1,
                           hermitian=True, orth="lanczos")
    r2 = krylov.pp_arnoldi(A.dot, b, -0.5, (0.37,), side="left", m_max=25, tol=0.0, k_chk=1,
                           hermitian=True, orth="lanczos")
    assert rel(r1["x"], r2["x"]) < 1e-12
    # H scales by c0^2
    assert np.allclose(r2["H"], 0.37 ** 2 * r1["H"], rtol=1e-10, atol=1e-12)


def test_left_equals_right_nonhermitian():
    dims = (8, 8, 8)
    A = ops.convdiff(dims, 0.5)
    b = synth.rhs(A.shape[0], 0)
    a, bb = ops.convdiff_interval(dims, 0.5)
    c = cheb.interp_coeffs(a, bb, 5)
    xs = exact.separable_fun(dims, b, 0.5, "convdiff", 0.5)
    for side in ("left", "right"):
        r = krylov.pp_arnoldi(A.dot, b, 0.5, c, (a, bb), side=side, m_max=120, tol=1e-12,
                              k_chk=4, hermitian=False, orth="cgs2")
        assert r["converged"] and rel(r["x"], xs) < 1e-10


def test_plain_reference_nonhermitian():
    dims = (10, 10, 10)
    A = ops.convdiff(dims, 0.5)
    b = synth.rhs(A.shape[0], 0)
    r = krylov.plain_reference(A.dot, b, -0.5, tol=1e-13, m_max=400, k_chk=8)
    assert rel(r["x"], exact.separable_fun(dims, b, -0.5, "convdiff", 0.5)) < 1e-11


def test_diagonal_lucky_breakdown():
    # P5: n distinct eigenvalues -> the Krylov space is exhausted at m = n, result exact
    n = 24
    a = np.linspace(0.5, 4.0, n)
    b = synth.rhs(n, 1)
    r = krylov.pp_arnoldi(lambda v: a * v, b, -0.5, (1.0,), m_max=60, tol=1e-30, k_chk=1,
                          hermitian=True, orth="cgs2")
    assert r["iters"] == n and r["converged"]
    assert rel(r["x"], a ** -0.5 * b) < 1e-11


def test_singular_semisimple_sqrt():
    # P6 / Thm. 4.1: periodic 2D Laplacian (eigenvalue 0 semi-simple); A^{1/2} b = A^{-1/2}(A b)
    N = 16
    T = ops.tridiag(N, -1.0, 2.0, -1.0).tolil()
    T[0, N - 1] = -1.0
    T[N - 1, 0] = -1.0
    A = ops.kron_sum([T.tocsr(), T.tocsr()])
    b = synth.rhs(N * N, 6)
    # Fourier closed form (numpy FFT as the library step)
    k = np.arange(N)
    l1 = 2 - 2 * np.cos(2 * np.pi * k / N)
    lam = l1[:, None] + l1[None, :]
    xs = np.real(np.fft.ifft2(np.sqrt(lam) * np.fft.fft2(b.reshape(N, N)))).reshape(-1)
    lo = 2 - 2 * np.cos(2 * np.pi / N)          # smallest nonzero eigenvalue
    c = cheb.interp_coeffs(lo, 8.0, 6)
    r = krylov.pp_arnoldi(A.dot, b, 0.5, c, (lo, 8.0), m_max=100, tol=1e-12, k_chk=2,
                          hermitian=True, orth="lanczos")
    assert r["converged"] and rel(r["x"], xs) < 1e-10


def test_mutation_is_caught():
    # a planted sign error in the oracle's q(A) (c_1 negated) breaks convergence to x*
    dims = (16, 16)
    A = ops.laplace(dims)
    b = synth.rhs(A.shape[0], 0)
    a, bb = ops.laplace_interval(dims)
    c = cheb.interp_coeffs(a, bb, 6)
    c_bad = c.copy()
    c_bad[1] = -c_bad[1]
    xs = exact.separable_fun(dims, b, -0.5)
    r = krylov.pp_arnoldi(A.dot, b, -0.5, c_bad, (a, bb), m_max=80, tol=1e-12, k_chk=2,
                          hermitian=True, orth="lanczos")
    assert rel(r["x"], xs) > 1e-6


def _table1():
    rows = []
    for line in open(os.path.join(GOLD, "table1_laplace3d_100.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append(tuple(int(v) for v in line.split()))
    return {r[0]: r[1:] for r in rows}


TAB1 = _table1()


@pytest.mark.parametrize("d", [pytest.param(1, marks=pytest.mark.slow),
                               pytest.param(4, marks=pytest.mark.slow), 8, 16])
def test_table1_counts(d):
    # P3: Table 1 iterations / mvms / inner products (right preconditioning, Lanczos, no reorth.)
    N = 100
    dims = (N, N, N)
    A = ops.laplace(dims)
    b = synth.rhs(A.shape[0], 0)
    b = b / np.linalg.norm(b)
    xs = exact.separable_fun(dims, b, -0.5)
    a, bb = ops.laplace_interval(dims)
    c = cheb.interp_coeffs(a, bb, d)
    r = krylov.pp_arnoldi(A.dot, b, -0.5, c, (a, bb), side="right", m_max=600, tol=1e-12,
                          k_chk=64 // d, hermitian=True, orth="lanczos", stop="true", exact=xs)
    assert (r["iters"], r["mvms"], r["inner_products"]) == TAB1[d]
