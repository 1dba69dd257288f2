"""Pins of the oracle's Chebyshev preconditioner (Sec. 5.1, Sec. 3.2 Example, Prop. 3.2)."""
import os

import numpy as np
import pytest

import synth
from oracle import chebyshev as cheb, exact, operators as ops

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, val, tol = line.split()[:3]
        out[key] = (float(val), float(tol))
    return out


def test_worked_example_sec32():
    # P2: 50 x 50 Laplacian, d = 32 (Sec. 3.2, Example)
    g = read_golden("e0_laplace2d_50.txt")
    dims = (50, 50)
    lam = exact.separable_eigs(dims)
    a, b = ops.laplace_interval(dims)
    kA = b / a
    assert abs(kA - g["kappa_A"][0]) < g["kappa_A"][1]
    c = cheb.interp_coeffs(a, b, 32)
    assert len(c) == 32
    eps = cheb.rel_error(c, a, b)
    assert abs(eps - g["eps"][0]) < g["eps"][1]
    pre = cheb.preconditioned_spectrum(c, a, b, lam)
    kpre = pre.max() / pre.min()
    assert abs(kpre - g["kappa_pre"][0]) < g["kappa_pre"][1]
    bound = cheb.kappa_pre_bound(eps)
    assert abs(bound - g["kappa_pre_bound"][0]) < g["kappa_pre_bound"][1]
    # Prop. 3.2 holds, and the spectrum sits inside [1-2e-e^2, 1+2e+e^2]
    assert kpre <= bound
    assert pre.min() >= 1 - 2 * eps - eps ** 2 - 1e-12 and pre.max() <= 1 + 2 * eps + eps ** 2 + 1e-12
    assert cheb.positive_on(c, a, b)


def test_truncated_series_reading_differs():
    # The exact-integral (truncated series) reading does not give the printed numbers.
    dims = (50, 50)
    a, b = ops.laplace_interval(dims)
    c = cheb.series_coeffs(a, b, 31)
    assert abs(cheb.rel_error(c, a, b) - 0.1263) > 0.03


def test_interpolates_at_nodes_and_reproduces_polynomials():
    a, b = 0.3, 7.0
    d = 9
    c = cheb.interp_coeffs(a, b, d)
    t = np.pi * (np.arange(d) + 0.5) / d
    z = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(t)
    assert np.allclose(cheb.q_eval(c, a, b, z), z ** -0.5, rtol=1e-14)
    # a polynomial of degree < d is reproduced exactly
    f = lambda x: 2.0 - 3.0 * x + 0.25 * x ** 3
    cp = cheb.interp_coeffs(a, b, d, f)
    zz = np.linspace(a, b, 50)
    assert np.allclose(cheb.q_eval(cp, a, b, zz), f(zz), rtol=1e-13, atol=1e-13)
    assert np.all(np.abs(cp[4:]) < 1e-13)


def test_series_coeffs_known_expansion():
    # 1/sqrt(z) on [a,b] is (x + s)^{-1/2} up to a constant, s = (b+a)/(b-a); its
    # Chebyshev coefficients are proportional to the toroidal functions Q_{i-1/2}(s),
    # asymptotically i^{-1/2} rho^{-i} with rho = s + sqrt(s^2-1) = (sqrt(k)+1)/(sqrt(k)-1)
    a, b = 1.0, 9.0
    c = cheb.series_coeffs(a, b, 40)
    kappa = b / a
    rho = (np.sqrt(kappa) + 1) / (np.sqrt(kappa) - 1)
    i = np.arange(10, 29)
    ratios = np.abs(c[i + 1] / c[i])
    assert np.allclose(ratios, np.sqrt((i - 0.5) / (i + 0.5)) / rho, rtol=5e-3)
    assert np.all(c * (-1.0) ** np.arange(41) > 0)  # singularity at the left end: alternating signs


@pytest.mark.parametrize("deg", [0, 1, 5, 12])
def test_q_apply_matches_spectral_definition(deg):
    dims = (9, 7)
    A = ops.laplace(dims)
    a, b = ops.laplace_interval(dims)
    c = cheb.interp_coeffs(a, b, deg + 1)
    v = synth.rhs(A.shape[0], 2)
    lam, U = np.linalg.eigh(A.toarray())
    ref = U @ (cheb.q_eval(c, a, b, lam) * (U.T @ v))
    got = cheb.q_apply(A.dot, c, a, b, v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


def test_mutation_is_caught():
    # planted mistake in the oracle's polynomial: dropping the last coefficient
    # or flipping the sign of one changes kappa_pre of the worked example
    dims = (50, 50)
    lam = exact.separable_eigs(dims)
    a, b = ops.laplace_interval(dims)
    c = cheb.interp_coeffs(a, b, 32)
    for bad in (c[:-1], c * np.where(np.arange(32) == 3, -1, 1)):
        pre = cheb.preconditioned_spectrum(bad, a, b, lam)
        assert abs(pre.max() / pre.min() - 1.5153) > 5e-5
