"""Chebyshev preconditioning polynomial q ~ z^{-1/2} on [a,b] (Sec. 5.1), FP64.

Test infrastructure only.

Degree convention: the paper's d is the number of nodes, q has degree d-1
(Sec. 6, Example 1 and Table 1 caption).  The library's `degree` k is
deg q, so d = k + 1.

Reading of the coefficient integrals (Sec. 5.1): the worked example of
Sec. 3.2 (50 x 50 Laplacian, d = 32, kappa_pre = 1.5153) is reproduced when
the integrals are evaluated with the d-point Gauss-Chebyshev rule, i.e. q is
the interpolant at the d first-kind Chebyshev nodes of [a,b].  That is the
default (`interp_coeffs`); `series_coeffs` evaluates the same integrals with
a fine M-point rule (the truncated series).
"""
import numpy as np


def sigma(z, a, b):
    """Affine map of [a,b] onto [-1,1]: T_i^{[a,b]}(z) = T_i(sigma(z))."""
    return (2.0 * z - (a + b)) / (b - a)


def _gauss_chebyshev_coeffs(f, a, b, M, ncoef):
    # c_i = (2/pi) int_a^b w(z) f(z) T_i^{[a,b]}(z) dz  (c_0 with 1/pi),
    # w(z) = ((z-a)(b-z))^{-1/2}; substituting z = (a+b)/2 + (b-a)/2 cos(t)
    # gives (2/pi) int_0^pi f(z(t)) cos(i t) dt, evaluated with the M-point
    # midpoint rule in t (= M-point Gauss-Chebyshev rule).
    t = np.pi * (np.arange(M) + 0.5) / M
    fz = f(0.5 * (a + b) + 0.5 * (b - a) * np.cos(t))
    i = np.arange(ncoef)
    c = (2.0 / M) * (np.cos(np.outer(i, t)) @ fz)
    c[0] *= 0.5
    return c


def interp_coeffs(a, b, d, f=lambda z: z ** -0.5):
    """Coefficients c_0..c_{d-1} of the degree d-1 interpolant at d first-kind nodes."""
    return _gauss_chebyshev_coeffs(f, a, b, d, d)


def series_coeffs(a, b, degree, M=4096, f=lambda z: z ** -0.5):
    """Coefficients c_0..c_degree of the truncated Chebyshev series (fine quadrature)."""
    return _gauss_chebyshev_coeffs(f, a, b, M, degree + 1)


def q_eval(c, a, b, z):
    """q(z) = sum_i c_i T_i(sigma(z)) for real z (numpy's chebval as the library step)."""
    return np.polynomial.chebyshev.chebval(sigma(np.asarray(z, dtype=np.float64), a, b), c)


def q_apply(matvec, c, a, b, v):
    """q(A) v by the definition sum_i c_i T_i(sigma(A)) v.

    T_0 v = v, T_1 v = sigma(A) v, T_{i+1} v = 2 sigma(A) T_i v - T_{i-1} v
    (three-term recurrence of the Chebyshev polynomials), accumulated term by
    term.  Uses len(c)-1 products with A.
    """
    def s_mv(x):
        return (2.0 * matvec(x) - (a + b) * x) / (b - a)

    t_prev = v
    y = c[0] * v
    if len(c) == 1:
        return y
    t_cur = s_mv(v)
    y = y + c[1] * t_cur
    for i in range(2, len(c)):
        t_next = 2.0 * s_mv(t_cur) - t_prev
        y = y + c[i] * t_next
        t_prev, t_cur = t_cur, t_next
    return y


def grid(a, b, npts=200001):
    """Evaluation grid on [a,b]: uniform plus geometric points (both include a, b)."""
    return np.unique(np.concatenate([np.linspace(a, b, npts), np.geomspace(a, b, npts)]))


def rel_error(c, a, b, npts=200001):
    """eps = max_{z in [a,b]} |1 - sqrt(z) q(z)|, the uniform relative error of Prop. 3.2."""
    z = grid(a, b, npts)
    return float(np.max(np.abs(1.0 - np.sqrt(z) * q_eval(c, a, b, z))))


def kappa_pre_bound(eps):
    """Prop. 3.2: kappa_pre <= (1 + 2 eps + eps^2) / (1 - 2 eps - eps^2) for eps < sqrt(2)-1."""
    if not eps < np.sqrt(2.0) - 1.0:
        return np.inf
    return (1.0 + 2.0 * eps + eps * eps) / (1.0 - 2.0 * eps - eps * eps)


def preconditioned_spectrum(c, a, b, eigs):
    """Eigenvalues lambda q(lambda)^2 of A q(A)^2 for Hermitian A with eigenvalues `eigs`."""
    eigs = np.asarray(eigs, dtype=np.float64)
    return eigs * q_eval(c, a, b, eigs) ** 2


def positive_on(c, a, b, npts=200001):
    """Numerical check (Sec. 5.1, last paragraph) that q > 0 on [a,b]."""
    return bool(np.min(q_eval(c, a, b, grid(a, b, npts))) > 0.0)


def image_interval(c, a, b, npts=200001):
    """[min, max] of z q(z)^2 over [a,b] (encloses spec(A q(A)^2) if spec(A) in [a,b])."""
    z = grid(a, b, npts)
    p = z * q_eval(c, a, b, z) ** 2
    return float(np.min(p)), float(np.max(p))
