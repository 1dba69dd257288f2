"""Polynomially preconditioned Arnoldi / Lanczos for A^{-1/2} b and A^{1/2} b, FP64.

Test infrastructure only.

* pp_arnoldi follows Algorithm 1 (left preconditioning, Sec. 3.1) and
  Algorithm 2 (right preconditioning) step by step: the preconditioned
  product is applied in three stages (A, then q(A) twice), never as a
  polynomial p = q^2; the basis is orthogonalized with the printed modified
  Gram-Schmidt loop (orth="mgs"), its Hermitian three-term specialization
  (orth="lanczos", Table 1 counts two inner products per iteration) or
  classical Gram-Schmidt applied twice (orth="cgs2", full
  reorthogonalization as used in Sec. 6, Example 3).
* f(H_m) e_1 uses a blocked Schur square root and a solve (Sec. 3.1, after
  Algorithm 1) for Hessenberg H; for the tridiagonal Lanczos matrix the
  eigendecomposition.
* A^{1/2} b is computed as A^{-1/2}(A b) (Sec. 4).
* Stopping (Sec. 6, Example 1): every k_chk iterations the relative norm of
  the difference of consecutive iterates ||f_m - f_{m+k}|| / ||f_{m+k}|| is
  formed; with left preconditioning it comes from the small coefficient
  vectors alone since V_m is orthonormal (Sec. 3.1).  stop="true" instead
  compares with a given exact solution (how Table 1 counts iterations).
"""
import numpy as np
import scipy.linalg as sla

from . import chebyshev as cheb


def fH_e1(H, beta, power=-0.5, hermitian=False):
    """z = beta * H^{power} e_1 for the small m x m Hessenberg / tridiagonal H.

    hermitian=True reads only the diagonal and sub-diagonal (symmetric
    tridiagonal Lanczos matrix).
    """
    m = H.shape[0]
    e1 = np.zeros(m, dtype=H.dtype)
    e1[0] = beta
    if hermitian:
        d = np.real(np.diag(H)).astype(np.float64)
        e = np.real(np.diag(H, -1)).astype(np.float64) if m > 1 else np.zeros(0)
        if m == 1:
            return np.array([beta * d[0] ** power], dtype=H.dtype)
        th, Q = sla.eigh_tridiagonal(d, e)
        return (Q @ (np.power(th, power) * (Q[0, :] * beta))).astype(H.dtype)
    S = sla.sqrtm(H)
    if power > 0:
        return S @ e1
    return np.linalg.solve(S, e1)


def pp_arnoldi(A_mv, b, power=-0.5, coeffs=(1.0,), ab=(0.0, 1.0), side="left",
               m_max=200, tol=1e-10, k_chk=1, hermitian=False, orth="mgs",
               stop="estimate", exact=None, breakdown_tol=1e-14, on_iter=None, q=None):
    """Polynomially preconditioned Arnoldi for A^{power} b, power = -1/2 or +1/2.

    coeffs, ab: Chebyshev coefficients of q and its interval (see
    oracle.chebyshev); coeffs=(1.0,) is q = 1, i.e. plain Arnoldi.
    q = (degree, q_mv), if given, replaces the Chebyshev q by another
    polynomial of that degree applied by q_mv(v) = q(A) v (Sec. 5.2).
    Returns a dict with the iterate x, the iteration count and the operation
    counters (mvms, inner products) in the sense of Tables 1-3.  on_iter(j), if
    given, is called after every iteration (a timing hook; no effect on results).
    """
    c = np.asarray(coeffs, dtype=np.float64)
    a, bb = ab
    deg = len(c) - 1 if q is None else q[0]
    mvms = 0
    ip = 0
    rhs = np.asarray(b)
    if power > 0:                        # Sec. 4: A^{1/2} b = A^{-1/2} (A b)
        rhs = A_mv(rhs)
        mvms += 1

    def q_mv(v):
        if q is not None:
            return q[1](v)
        return cheb.q_apply(A_mv, c, a, bb, v)

    n = rhs.shape[0]
    dt = np.result_type(rhs.dtype, np.float64)
    V = np.zeros((m_max + 1, n), dtype=dt)
    Y = np.zeros((m_max, n), dtype=dt) if side == "right" else None
    H = np.zeros((m_max + 1, m_max), dtype=dt)

    if side == "left":                   # Algorithm 1: start from c = q(A) b
        start = q_mv(rhs)
        mvms += deg
    else:                                # Algorithm 2: start from b
        start = rhs
    beta = np.linalg.norm(start)         # not counted: Tables 1-3 count the loop only
    V[0] = start / beta

    # The tridiagonal eigensolver is used for the three-term recurrence only;
    # a Gram-Schmidt H is treated as a full Hessenberg matrix.
    tridiag = hermitian and orth == "lanczos"
    history = []
    z_prev = None
    x = None
    m = 0
    converged = False
    if on_iter is not None:
        on_iter(-1)
    for j in range(m_max):
        if side == "left":               # Algorithm 1: u = A v_j, y = q(A) u, w = q(A) y
            u = A_mv(V[j])
            y = q_mv(u)
            w = q_mv(y)
        else:                            # Algorithm 2: y_j = q(A) v_j, u = q(A) y_j, w = A u
            Y[j] = q_mv(V[j])
            u = q_mv(Y[j])
            w = A_mv(u)
        mvms += 2 * deg + 1

        if orth == "mgs":                # the modified Gram-Schmidt loop as printed
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - V[i] * H[i, j]
            ip += j + 1
        elif orth == "lanczos":          # Hermitian: only v_{j-1}, v_j are needed
            if j > 0:
                H[j - 1, j] = np.conj(H[j, j - 1])
                w = w - V[j - 1] * H[j - 1, j]
            H[j, j] = np.vdot(V[j], w)
            w = w - V[j] * H[j, j]
            ip += 1
        elif orth == "cgs2":
            for _ in range(2):
                h = V[: j + 1].conj() @ w
                w = w - V[: j + 1].T @ h
                H[: j + 1, j] += h
            ip += 2 * (j + 1)
        else:
            raise ValueError(orth)

        hn = np.linalg.norm(w)           # h_{j+1,j} = ||w||
        ip += 1
        H[j + 1, j] = hn
        m = j + 1
        scale = np.linalg.norm(H[: j + 2, j])
        lucky = hn <= breakdown_tol * max(scale, 1e-300)
        if not lucky:
            V[j + 1] = w / hn            # v_{j+1} = w / h_{j+1,j}
        if on_iter is not None:
            on_iter(j)

        if lucky or m % k_chk == 0 or m == m_max:
            z = fH_e1(H[:m, :m], beta, -0.5, tridiag)
            basis = V[:m] if side == "left" else Y[:m]
            if stop == "true" or side == "right" or z_prev is None:
                x = basis.T @ z
            if stop == "true":
                est = np.linalg.norm(x - exact) / np.linalg.norm(exact)
            elif z_prev is None:
                est = np.inf
            else:
                zp = np.zeros(z.shape, dtype=np.result_type(z, z_prev))
                zp[: z_prev.shape[0]] = z_prev
                if side == "left":
                    est = np.linalg.norm(zp - z) / np.linalg.norm(z)
                else:
                    est = np.linalg.norm(basis.T @ (zp - z)) / np.linalg.norm(x)
            history.append((m, est))
            z_prev = z
            if lucky or est < tol:
                converged = True
                break
    basis = V[:m] if side == "left" else Y[:m]
    z = fH_e1(H[:m, :m], beta, -0.5, tridiag)
    x = basis.T @ z
    return dict(x=x, iters=m, mvms=mvms, inner_products=ip, converged=converged,
                history=history, H=H[: m + 1, :m], beta=beta)


def plain_reference(A_mv, b, power=-0.5, tol=1e-13, m_max=2000, k_chk=8, hermitian=False):
    """Unpreconditioned Arnoldi with full reorthogonalization (CGS2) to a tight tolerance.

    The large-n stand-in for the exact solution, as the paper does with a
    tighter-tolerance run (Sec. 6, Examples 2 and 3).
    """
    return pp_arnoldi(A_mv, b, power, coeffs=(1.0,), side="left", m_max=m_max, tol=tol,
                      k_chk=k_chk, hermitian=hermitian, orth="cgs2")
