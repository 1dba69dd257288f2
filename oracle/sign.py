"""Matrix sign function sign(Q) b = Q (Q^2)^{-1/2} b (Sec. 6, Example 2), FP64 / complex128.

Test infrastructure only.

* sign_krylov: (Q^2)^{-1/2} b by the polynomially preconditioned Arnoldi
  method of oracle.krylov on the operator Q^2, applied as two products with
  Q (Q^2 is never formed), then one more product with Q.
* sign_dense: the definition for a diagonalizable Q = X diag(lambda) X^{-1}
  with no eigenvalue on the imaginary axis: sign(Q) = X diag(sign(Re
  lambda)) X^{-1}, equal to Q (Q^2)^{-1/2} with the principal square root.
* overlap_apply: D_ov b = b + rho Gamma_5 sign(Q) b (the overlap operator of
  Sec. 6, Example 2, for a given sign(Q) b).
"""
import numpy as np

from . import krylov


def sign_krylov(Q_mv, b, **kw):
    """sign(Q) b and the pp_arnoldi result dict for (Q^2)^{-1/2} b (kw go to pp_arnoldi)."""
    r = krylov.pp_arnoldi(lambda v: Q_mv(Q_mv(v)), b, -0.5, **kw)
    return Q_mv(r["x"]), r


def sign_dense(Q):
    lam, X = np.linalg.eig(np.asarray(Q, dtype=np.complex128))
    return (X * np.sign(lam.real)) @ np.linalg.inv(X)


def overlap_apply(b, sign_b, rho):
    s = np.asarray(sign_b).reshape(-1, 4, 3).copy()
    s[:, 2:] *= -1.0
    return np.asarray(b) + rho * s.reshape(-1)
