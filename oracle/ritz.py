"""Preconditioning polynomials interpolating z^{-1/2} at Ritz or harmonic
Ritz values (Sec. 5.2), FP64.

Test infrastructure only.

* arnoldi: d steps of the Arnoldi process from a given start vector, each
  new vector orthogonalized by classical Gram-Schmidt applied twice;
  returns the (d+1) x d Hessenberg matrix H.  For Hermitian A it is
  tridiagonal up to rounding, and the Hermitian reading below takes its
  diagonal and sub-diagonal (the Lanczos matrix T_d).
* ritz_values: the eigenvalues of H_d (the leading d x d block); Hermitian:
  of T_d.
* harmonic_ritz_values: the eigenvalues of H_d + h_{d+1,d}^2 H_d^{-*} e_d e_d^*
  (the matrix of Sec. 5.2); Hermitian: of T_d + beta_d^2 T_d^{-1} e_d e_d^T,
  which is real-diagonalizable for positive definite T_d.
* leja_order: Leja ordering: first a node of largest modulus, then each time
  the remaining node with the largest product of distances to the nodes
  already taken (ties: the earliest in the input order); complex nodes of a
  real problem come in conjugate pairs, each pair kept adjacent.
* newton_coeffs / newton_eval / newton_apply: q of degree d-1 interpolating
  f at the ordered nodes, in Newton form
      q(z) = sum_{i<d} a_i prod_{k<i} (z - x_k),  a_i = f[x_0, ..., x_i],
  the divided differences; evaluated here term by term, straight from that
  definition (the library uses a Horner scheme, as Sec. 5.2 does).
* start_vector: the fixed pseudo-random start of the library's Arnoldi run:
  entry i is (s_i >> 11) 2^-52 - 1, s_i the SplitMix64 output (Steele, Lea,
  Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) for
  the state seed + (i + 1) * 0x9E3779B97F4A7C15, implemented here from that
  published definition.  A complex vector of n entries takes the 2n values
  as (real, imaginary) pairs.
"""
import numpy as np

_M64 = (1 << 64) - 1
LIBRARY_SEED = 0x5EED


def splitmix64(seed, i):
    """SplitMix64 output for the state seed + (i + 1) * 0x9E3779B97F4A7C15 (exact integers)."""
    z = (seed + 0x9E3779B97F4A7C15 * (i + 1)) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def start_values(count, seed=LIBRARY_SEED):
    """(splitmix64(seed, i) >> 11) * 2^-52 - 1 for i < count, in [-1, 1)."""
    i = np.arange(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.uint64(0x9E3779B97F4A7C15) * (i + np.uint64(1))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0


def start_vector(n, complex_=False, seed=LIBRARY_SEED):
    if complex_:
        r = start_values(2 * n, seed)
        return r[0::2] + 1j * r[1::2]
    return start_values(n, seed)


def arnoldi(A_mv, v0, d):
    """d Arnoldi steps (CGS2) from v0: H ((m+1) x m) and the basis V ((m+1) x n).

    Stops early (m < d) if h_{j+1,j} vanishes to rounding (an invariant
    subspace); then H is m x m plus a zero row.
    """
    v = np.asarray(v0)
    dt = np.result_type(v.dtype, np.float64)
    V = np.zeros((d + 1, v.shape[0]), dtype=dt)
    H = np.zeros((d + 1, d), dtype=dt)
    V[0] = v / np.linalg.norm(v)
    m = d
    for j in range(d):
        w = A_mv(V[j])
        for _ in range(2):
            h = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h
            H[: j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * np.linalg.norm(H[: j + 2, j]):
            H[j + 1, j] = 0.0
            m = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return H[: m + 1, :m], V[: m + 1]


def tridiag_of(H):
    """The Lanczos matrix read from a Hermitian Arnoldi H: diagonal and sub-diagonal, symmetric."""
    m = H.shape[1]
    al = np.real(np.diag(H[:m, :m]))
    be = np.real(np.diag(H, -1))  # beta_1 .. beta_m (beta_m = h_{m+1,m})
    T = np.diag(al) + np.diag(be[: m - 1], 1) + np.diag(be[: m - 1], -1)
    return T, (be[m - 1] if H.shape[0] > m else 0.0)


def ritz_values(H, hermitian=True):
    if hermitian:
        T, _ = tridiag_of(H)
        return np.linalg.eigvalsh(T)
    m = H.shape[1]
    return np.linalg.eigvals(H[:m, :m])


def harmonic_ritz_values(H, hermitian=True):
    m = H.shape[1]
    e = np.zeros(m)
    e[-1] = 1.0
    if hermitian:
        T, beta = tridiag_of(H)
        Ht = T + beta ** 2 * np.outer(np.linalg.solve(T, e), e)
        return np.sort(np.real(np.linalg.eigvals(Ht)))
    Hd = H[:m, :m]
    h = H[m, m - 1] if H.shape[0] > m else 0.0
    Ht = Hd + abs(h) ** 2 * np.outer(np.linalg.solve(Hd.conj().T, e), e)
    return np.linalg.eigvals(Ht)


def leja_order(nodes, pairs=True):
    """Leja order; real input gives a real array.

    Complex nodes with pairs=True (conjugate pairs of a real problem): the
    candidates are the nodes with Im >= 0; a chosen complex node is followed
    at once by its conjugate, so every pair is adjacent (a conjugation-closed
    node set after each pair).  pairs=False (a complex problem, nodes without
    that symmetry): every node is a candidate on its own.
    """
    arr = np.asarray(nodes)
    real = not np.iscomplexobj(arr) or np.all(arr.imag == 0)
    if real:
        rest = [complex(x) for x in np.real(arr).astype(np.float64)]
    elif pairs:
        rest = [complex(x) for x in arr if x.imag >= 0]
    else:
        rest = [complex(x) for x in arr]
    first = max(range(len(rest)), key=lambda i: (abs(rest[i]), -i))
    out = []

    def take(z):
        out.append(z)
        if pairs and z.imag > 0:
            out.append(z.conjugate())

    take(rest.pop(first))

    def logprod(z):
        return sum(np.log(abs(z - x)) if z != x else -np.inf for x in out)

    while rest:
        scores = [logprod(z) for z in rest]
        best = int(np.argmax(scores))  # first maximum
        take(rest.pop(best))
    out = np.array(out)
    return out.real.copy() if real else out


def _dtype(x):
    return np.complex128 if np.iscomplexobj(x) else np.float64


def newton_coeffs(nodes, f=lambda z: z ** -0.5):
    """a_i = f[x_0, ..., x_i] from the recursive divided-difference table
    (complex for complex nodes; f(z) = z^{-1/2} on the principal branch)."""
    x = np.asarray(nodes)
    x = x.astype(_dtype(x))
    d = len(x)
    col = np.asarray(f(x), dtype=x.dtype)
    a = [col[0]]
    for k in range(1, d):
        col = (col[1:] - col[:-1]) / (x[k:] - x[:-k])
        a.append(col[0])
    return np.array(a)


def newton_eval(a, nodes, z):
    a = np.asarray(a)
    z = np.asarray(z)
    dt = np.result_type(a.dtype, np.asarray(nodes).dtype, z.dtype, np.float64)
    z = z.astype(dt)
    out = np.zeros_like(z)
    prod = np.ones_like(z)
    for i in range(len(a)):
        out = out + a[i] * prod
        prod = prod * (z - nodes[i])
    return out


def newton_apply(A_mv, a, nodes, v):
    """q(A) v = sum_i a_i prod_{k<i} (A - x_k I) v, term by term (complex
    arithmetic when the nodes are complex; a real q of a real A gives a real
    result up to rounding, returned as its real part for real v)."""
    v = np.asarray(v)
    dt = np.result_type(v.dtype, np.asarray(a).dtype, np.asarray(nodes).dtype, np.float64)
    out = np.zeros(v.shape, dtype=dt)
    p = v.astype(dt)
    for i in range(len(a)):
        out = out + a[i] * p
        if i + 1 < len(a):
            p = A_mv(p) - nodes[i] * p
    if not np.iscomplexobj(v) and np.iscomplexobj(out):
        return out.real.copy()
    return out


def ritz_poly(A_mv, n, degree, harmonic=False, complex_=False, hermitian=True):
    """Leja-ordered nodes and Newton coefficients of q, deg q = degree, from
    degree + 1 Arnoldi steps on the library's start vector.

    Hermitian A: real nodes.  Real non-Hermitian A: the eigenvalues of H_d
    (or of the harmonic matrix), complex ones in conjugate pairs.  Complex
    non-Hermitian A (complex_ and not hermitian): the eigenvalues of the
    complex H_d, Leja-ordered one by one (no conjugate symmetry).
    Returns (nodes, coeffs); fewer nodes if the Krylov space became invariant.
    """
    H, _ = arnoldi(A_mv, start_vector(n, complex_), degree + 1)
    th = harmonic_ritz_values(H, hermitian) if harmonic else ritz_values(H, hermitian)
    if complex_ and not hermitian:
        x = leja_order(np.asarray(th, dtype=np.complex128), pairs=False)
    elif hermitian or np.all(np.abs(np.imag(th)) == 0):
        x = leja_order(np.sort(np.real(th)))
    else:
        # snap the conjugate pairs of the real H_d exactly (eigvals returns them
        # conjugate to rounding) and order the set
        th = np.asarray(th)
        up = th[th.imag > 0]
        re = np.real(th[th.imag == 0])
        x = leja_order(np.concatenate([re, up, up.conj()]))
    return x, newton_coeffs(x)
