"""Exact x* = A^{-1/2} b and A^{1/2} b by plain definitions (test infrastructure only).

The preconditioned method converges to the principal (inverse) square root
(Sec. 3, branch discussion around Eq. (3.4)), so the oracle of the final
result is that definition, never the method:

* dense_fun:     Hermitian A -> eigh; general A -> Schur square root
                 (scipy.linalg.sqrtm, the blocked Schur method named in
                 Sec. 3.1) followed by a solve for the inverse root.
* separable_fun: operators that are Kronecker sums of 1D factors with a
                 closed-form eigen-decomposition (Dirichlet Laplacian;
                 convection-diffusion through the diagonal similarity of
                 oracle.operators.convdiff_eigs_1d).
* diagonal_fun:  diagonal A.

`power` is -0.5 (INVSQRT) or +0.5 (SQRT).
"""
import numpy as np
import scipy.linalg as sla

from . import operators as ops


def _fscalar(lam, power):
    return np.power(lam.astype(np.complex128) if np.iscomplexobj(lam) else lam, power)


def dense_fun(A, b, power, hermitian=None):
    """f(A) b for a dense (or sparse, converted) matrix of modest size."""
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    if hermitian is None:
        hermitian = np.allclose(A, A.conj().T, rtol=0, atol=0)
    if hermitian:
        lam, U = np.linalg.eigh(A)
        if np.any(lam <= 0) and power < 0:
            raise ValueError("A must be positive definite for A^{-1/2}")
        lam = np.maximum(lam, 0.0)
        return U @ (np.power(lam, power) * (U.conj().T @ b))
    S = sla.sqrtm(A)
    if power > 0:
        return S @ b
    return np.linalg.solve(S, b)


def _apply_along(mats, X):
    """Apply mats[d] along grid axis d (d = 0 is the fastest index)."""
    nd = len(mats)
    for d, M in enumerate(mats):
        ax = nd - 1 - d  # C-order array: the fastest index is the last axis
        X = np.moveaxis(np.tensordot(M, X, axes=([1], [ax])), 0, ax)
    return X


def separable_fun(dims, b, power, kind="laplace", ch=0.0):
    """Closed-form f(A) b for A = sum_d T_d with T_d = D S diag(l) S D^{-1}.

    Laplacian: D = I, S = sine basis, l = 2 - 2 cos(k pi/(N+1)).
    Convection-diffusion: D = diag((1+ch)^{j/2}), same S, shifted l.
    f(A) b = (D x S)(x ...) f(sum of l) (S x ...)(D^{-1} x ...) b.
    Exact to rounding for the Laplacian at any size; for convection-
    diffusion the similarity has condition (1+ch)^{(N-1)/2} per direction,
    so it is usable only for small N.
    """
    dims = tuple(int(N) for N in dims)
    shape = tuple(reversed(dims))  # C-order array with x fastest
    X = np.asarray(b, dtype=np.float64).reshape(shape)
    Ss = [ops.sine_basis(N) for N in dims]
    if kind == "laplace":
        ls = [ops.laplace_eigs_1d(N) for N in dims]
        Ds = None
    elif kind == "convdiff":
        ls = [ops.convdiff_eigs_1d(N, ch) for N in dims]
        r = np.sqrt(1.0 + ch)
        Ds = [r ** np.arange(1, N + 1) for N in dims]
    else:
        raise ValueError(kind)
    if Ds is not None:
        X = _apply_along([np.diag(1.0 / D) for D in Ds], X)
    X = _apply_along([S.T for S in Ss], X)
    lam = np.zeros(shape)
    for d, l in enumerate(ls):
        ax = len(dims) - 1 - d
        sh = [1] * len(dims)
        sh[ax] = dims[d]
        lam = lam + l.reshape(sh)
    X = X * np.power(lam, power)
    X = _apply_along(Ss, X)
    if Ds is not None:
        X = _apply_along([np.diag(D) for D in Ds], X)
    return X.reshape(-1)


def separable_eigs(dims, kind="laplace", ch=0.0):
    """All eigenvalues of the separable operator (unsorted, grid order)."""
    dims = tuple(int(N) for N in dims)
    shape = tuple(reversed(dims))
    lam = np.zeros(shape)
    for d, N in enumerate(dims):
        l = ops.laplace_eigs_1d(N) if kind == "laplace" else ops.convdiff_eigs_1d(N, ch)
        sh = [1] * len(dims)
        sh[len(dims) - 1 - d] = N
        lam = lam + l.reshape(sh)
    return lam.reshape(-1)


def diagonal_fun(a, b, power):
    """x*_i = a_i^power b_i for A = diag(a)."""
    return np.power(np.asarray(a, dtype=np.float64), power) * np.asarray(b)
