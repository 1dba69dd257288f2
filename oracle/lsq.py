"""Preconditioning polynomial by error minimization on a contour (Sec. 5.3), FP64.

Test infrastructure only.

q of degree d-1 minimizes sum_i |z_i^{-1/2} - q(z_i)|^2 over points
z_1..z_N discretizing a contour Gamma around the spectrum (Sec. 5.3):

* basis(z, d): the Arnoldi process on diag(z_1, ..., z_N) from the vector of
  ones / sqrt(N) (modified Gram-Schmidt, plain complex arithmetic) gives
  orthonormal basis polynomials p_0..p_{d-1} for the discrete inner product
  <p1, p2> = sum_i p1(z_i) conj(p2(z_i)) as the columns of P (their values at
  the points) and the Hessenberg matrix H with z P[:, :d-1] = P H.
* coeffs(P, f): alpha = P^* f (the columns are orthonormal), f = z^{-1/2}.
* evaluate(H, alpha, N, z): q(z) = sum_j alpha_j p_j(z), the p_j from the
  Arnoldi recurrence p_k = (z p_{k-1} - sum_{j<=k} h_{jk} p_{j-1}) / h_{k+1,k}.
* apply(A_mv, H, alpha, N, v): q(A) v by the same recurrence on vectors
  (d-1 products with A, no inner products), the evaluation Sec. 5.3 uses.
* contour(ritz, r_min, npts): a discretized contour from Ritz values: their
  convex hull (made symmetric about the real axis for a real problem), the
  parts closer to 0 than r_min replaced by the arc of radius r_min, points at
  equal arc length; all-real Ritz values give the segment
  [max(min, r_min), max].
"""
import numpy as np


def basis(z, d):
    z = np.asarray(z, dtype=np.complex128)
    N = z.shape[0]
    P = np.zeros((N, d), dtype=np.complex128)
    H = np.zeros((d, max(d - 1, 0)), dtype=np.complex128)
    P[:, 0] = 1.0 / np.sqrt(N)
    for k in range(1, d):
        w = z * P[:, k - 1]
        for j in range(k):
            H[j, k - 1] = np.vdot(P[:, j], w)
            w = w - H[j, k - 1] * P[:, j]
        H[k, k - 1] = np.linalg.norm(w)
        P[:, k] = w / H[k, k - 1]
    return P, H


def coeffs(P, f):
    return P.conj().T @ np.asarray(f, dtype=np.complex128)


def evaluate(H, alpha, N, z):
    z = np.asarray(z, dtype=np.complex128)
    d = len(alpha)
    p = [np.full(z.shape, 1.0 / np.sqrt(N), dtype=np.complex128)]
    for k in range(1, d):
        w = z * p[k - 1]
        for j in range(k):
            w = w - H[j, k - 1] * p[j]
        p.append(w / H[k, k - 1])
    return sum(alpha[j] * p[j] for j in range(d))


def apply(A_mv, H, alpha, N, v):
    """q(A) v by the basis recurrence; real for real A, v and a real q (returned as real)."""
    v = np.asarray(v)
    d = len(alpha)
    w = [v.astype(np.complex128) / np.sqrt(N)]
    for k in range(1, d):
        t = A_mv(w[k - 1])
        for j in range(k):
            t = t - H[j, k - 1] * w[j]
        w.append(t / H[k, k - 1])
    out = sum(alpha[j] * w[j] for j in range(d))
    if not np.iscomplexobj(v):
        return out.real.copy()
    return out


def _upper_chain(pts):
    """Upper convex hull of points symmetric about the real axis, from the
    right end of its intersection with the real axis to the left end:
    (max Re, 0), the hull vertices with Im > 0 right to left, (min Re, 0)."""
    P = sorted(set((float(p.real), float(p.imag)) for p in pts))
    up = []
    for p in reversed(P):  # monotone chain, right to left, counter-clockwise turns only
        while len(up) >= 2 and (up[-1][0] - up[-2][0]) * (p[1] - up[-2][1]) - \
                (up[-1][1] - up[-2][1]) * (p[0] - up[-2][0]) <= 0:
            up.pop()
        up.append(p)
    xs = [p[0] for p in P]
    chain = [complex(max(xs), 0.0)] + [complex(*p) for p in up if p[1] > 0] + [complex(min(xs), 0.0)]
    return np.array(chain)


def contour(ritz, r_min, npts):
    th = np.asarray(ritz, dtype=np.complex128)
    if np.all(th.imag == 0):
        lo, hi = max(th.real.min(), r_min), th.real.max()
        return np.linspace(lo, hi, npts).astype(np.complex128)
    chain = _upper_chain(np.concatenate([th, th.conj()]))
    # densely resampled, points inside the disc |z| < r_min pushed out radially
    # onto its circle (the part of the curve there becomes the arc)
    seg = np.abs(np.diff(chain))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    keep = seg > 0
    t = np.linspace(0.0, s[-1], 40 * npts)
    k = np.clip(np.searchsorted(s, t, side="right") - 1, 0, len(seg) - 1)
    while not np.all(keep[k]):  # skip zero-length pieces
        k = np.where(keep[k], k, k + 1)
    dense = chain[k] + (chain[k + 1] - chain[k]) * ((t - s[k]) / seg[k])
    small = np.abs(dense) < r_min
    dense[small] = r_min * dense[small] / np.abs(dense[small])
    # npts/2 points at equal arc length on the modified upper curve, mirrored
    arc = np.concatenate([[0.0], np.cumsum(np.abs(np.diff(dense)))])
    m = npts // 2
    tt = np.linspace(0.0, arc[-1], m)
    half = np.interp(tt, arc, dense.real) + 1j * np.interp(tt, arc, dense.imag)
    half[0] = half[0].real
    half[-1] = half[-1].real
    return np.concatenate([half, half[1:-1].conj()])
