"""Sparse FP64 test operators (oracle side; test infrastructure only).

Grid vectors are ordered with the x index fastest:
    idx = (k * Ny + j) * Nx + i.
Every operator is a Kronecker sum of 1D tridiagonal factors, one per grid
direction, unscaled (the h^2-scaled difference operator):

* Dirichlet Laplacian (Sec. 6, Example 1; Sec. 3.2 Example): factor
  tridiag(-1, 2, -1); the 2D/3D operators have diagonal 4/6.
* Upwind convection-diffusion -Lap(u) + c.grad(u), c = (c,c,c), c > 0, h^2-
  scaled with ch = c*h: factor tridiag(-(1+ch), 2+ch, -1) with the
  -(1+ch) entry on the sub-diagonal (the upwind neighbour i-1).  This
  operator is not in the paper; it is the non-Hermitian stand-in for the
  nonsymmetric examples of Sec. 6.
"""
import numpy as np
import scipy.sparse as sp


def tridiag(N, sub, diag, sup):
    """N x N tridiagonal CSR matrix with constant diagonals."""
    return sp.diags([np.full(N - 1, float(sub)), np.full(N, float(diag)),
                     np.full(N - 1, float(sup))], [-1, 0, 1], format="csr")


def kron_sum(factors):
    """Kronecker sum of 1D factors; factors[0] acts on the fastest index.

    A = sum_d I x ... x T_d x ... x I  with T_d at the position of dimension d
    (slowest dimension leftmost in the Kronecker products).
    """
    dims = [f.shape[0] for f in factors]
    n = int(np.prod(dims))
    A = sp.csr_matrix((n, n))
    for d, T in enumerate(factors):
        term = None
        # build from the slowest dimension to the fastest one
        for e in reversed(range(len(dims))):
            M = T if e == d else sp.identity(dims[e], format="csr")
            term = M if term is None else sp.kron(term, M, format="csr")
        A = A + term
    return A.tocsr()


def laplace_factor(N):
    return tridiag(N, -1.0, 2.0, -1.0)


def convdiff_factor(N, ch):
    return tridiag(N, -(1.0 + ch), 2.0 + ch, -1.0)


def laplace(dims):
    """Dirichlet Laplacian on a grid with `dims` = (Nx, Ny[, Nz]) interior points."""
    return kron_sum([laplace_factor(N) for N in dims])


def convdiff(dims, ch):
    """Upwind convection-diffusion operator with convection (c,c,c), c*h = ch."""
    return kron_sum([convdiff_factor(N, ch) for N in dims])


# ---- closed-form 1D eigen-decompositions ---------------------------------

def sine_basis(N):
    """Orthonormal eigenvectors of tridiag(-1,2,-1): S_jk = sqrt(2/(N+1)) sin(jk pi/(N+1))."""
    j = np.arange(1, N + 1)
    return np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(j, j) * np.pi / (N + 1))


def laplace_eigs_1d(N):
    """Eigenvalues 2 - 2 cos(k pi/(N+1)), k = 1..N, in the order of sine_basis's columns."""
    k = np.arange(1, N + 1)
    return 2.0 - 2.0 * np.cos(k * np.pi / (N + 1))


def convdiff_eigs_1d(N, ch):
    """Eigenvalues of tridiag(-(1+ch), 2+ch, -1).

    With D = diag(r^j), r = sqrt(1+ch), the factor equals D T_s D^{-1},
    T_s = tridiag(-r, 2+ch, -r) symmetric with the sine eigenvectors, so the
    eigenvalues are (2+ch) - 2 r cos(k pi/(N+1)).
    """
    k = np.arange(1, N + 1)
    return (2.0 + ch) - 2.0 * np.sqrt(1.0 + ch) * np.cos(k * np.pi / (N + 1))


def laplace_interval(dims):
    """Exact spectral interval of the Dirichlet Laplacian (Sec. 6, Example 1, for 3D)."""
    lo = sum(2.0 - 2.0 * np.cos(np.pi / (N + 1)) for N in dims)
    hi = sum(2.0 - 2.0 * np.cos(N * np.pi / (N + 1)) for N in dims)
    return lo, hi


def convdiff_interval(dims, ch):
    lo = sum(convdiff_eigs_1d(N, ch)[0] for N in dims)
    hi = sum(convdiff_eigs_1d(N, ch)[-1] for N in dims)
    return lo, hi
