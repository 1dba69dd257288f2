"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only (random right-hand sides, the CSR
arrays of the stencil test matrices, problem lists); none of the method's
arithmetic lives here.

Recipes
* b ~ N(0,1), FP64, numpy.random.default_rng(seed).standard_normal; seed 0
  for single problems, 1000 + i for the i-th problem of a batch.  The paper
  draws b at random (Sec. 6, Examples 1-3); relative errors do not depend on
  the scale of b.
* Stencil matrices in CSR with the grid ordering idx = (k*Ny + j)*Nx + i
  (x fastest); neighbours listed in increasing column order.
"""
import numpy as np


def rhs(n, seed=0, nrhs=1):
    """FP64 right-hand side(s): shape (n,) or, for nrhs > 1, (nrhs, n) (one row per RHS)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.standard_normal(n)
    return rng.standard_normal((nrhs, n))


def stencil_coeffs(kind, ch=0.0):
    """(diag, [(axis, offset, value), ...]) of the constant-coefficient stencils.

    laplace2d5 / laplace3d7: diagonal 4 / 6, every neighbour -1.
    convdiff3d7: diagonal 6 + 3 ch, upwind neighbours (offset -1) -(1 + ch),
    downwind neighbours (offset +1) -1.
    """
    if kind == "laplace2d5":
        return 4.0, [(ax, o, -1.0) for ax in range(2) for o in (-1, 1)]
    if kind == "laplace3d7":
        return 6.0, [(ax, o, -1.0) for ax in range(3) for o in (-1, 1)]
    if kind == "convdiff3d7":
        return 6.0 + 3.0 * ch, [(ax, o, (-(1.0 + ch) if o < 0 else -1.0))
                                for ax in range(3) for o in (-1, 1)]
    raise ValueError(kind)


def stencil_csr(kind, dims, ch=0.0):
    """CSR arrays (rowptr int64, col int32, val float64) of a stencil on a Dirichlet grid."""
    dims = tuple(int(N) for N in dims)
    diag, nbrs = stencil_coeffs(kind, ch)
    nd = len(dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for N in dims:
        coords.append(rem % N)
        rem //= N
    strides = [1]
    for N in dims[:-1]:
        strides.append(strides[-1] * N)
    rows, cols, vals = [idx], [idx], [np.full(n, diag)]
    for ax, off, v in nbrs:
        ok = (coords[ax] + off >= 0) & (coords[ax] + off < dims[ax])
        r = idx[ok]
        rows.append(r)
        cols.append(r + off * strides[ax])
        vals.append(np.full(r.shape[0], v))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals.astype(np.float64)


# ---- lattice gauge fields (Wilson operator inputs) ------------------------

def haar_su3(count, rng):
    """`count` Haar-distributed SU(3) matrices, complex128, shape (count, 3, 3).

    Mezzadri's method ("How to generate random matrices from the classical
    compact groups", Notices AMS 54, 2007): QR of a complex Ginibre matrix
    with the phases of R's diagonal moved into Q gives Haar U(3); dividing by
    a cube root of the determinant keeps left invariance and lands in SU(3).
    """
    Z = (rng.standard_normal((count, 3, 3)) + 1j * rng.standard_normal((count, 3, 3))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=1, axis2=2)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q * np.exp(-1j * np.angle(det) / 3.0)[:, None, None]


def wilson_links(dims, seed=1):
    """Gauge links U_mu(x) for a periodic 4D lattice, dims = (Lx, Ly, Lz, Lt).

    complex64 array of shape (V, 4, 3, 3), V = Lx Ly Lz Lt, site index
    s = ((t Lz + z) Ly + y) Lx + x, entry [s, mu, a, b] = U_mu(s)_{ab};
    Haar SU(3) matrices rounded to complex64 (both sides use the rounded
    values, so the operator is exactly the same on both).
    """
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    return haar_su3(4 * V, rng).reshape(V, 4, 3, 3).astype(np.complex64)


def unit_links(dims):
    """The free field U_mu(x) = 1 (complex64, layout of wilson_links)."""
    V = int(np.prod(dims))
    return np.broadcast_to(np.eye(3, dtype=np.complex64), (V, 4, 3, 3)).copy()


def spinor_field(dims, seed=0):
    """Random complex right-hand side b ~ N(0,1) + i N(0,1), 12 complex per site, complex128 (12 V,)."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    return rng.standard_normal(12 * V) + 1j * rng.standard_normal(12 * V)


# ---- batched workload (many independent problems) --------------------------

def batch_problems(count=64, seed=2, n_lo=1e3, n_hi=1e6, max_rhs=16):
    """Problem list of a batched run: dicts with kind ('laplace2d5',
    'laplace3d7' or 'convdiff3d7', uniform), dims (n log-uniform in
    [n_lo, n_hi], rounded to a square / cubic grid), nrhs ~ U{1..max_rhs}
    and f (+1 square root / -1 inverse square root, uniform)."""
    rng = np.random.default_rng(seed)
    kinds = ["laplace2d5", "laplace3d7", "convdiff3d7"]
    out = []
    for _ in range(count):
        kind = kinds[rng.integers(3)]
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        if kind == "laplace2d5":
            N = max(2, int(round(n ** 0.5)))
            dims = (N, N)
        else:
            N = max(2, int(round(n ** (1.0 / 3.0))))
            dims = (N, N, N)
        out.append({"kind": kind, "dims": dims, "nrhs": int(rng.integers(1, max_rhs + 1)),
                    "f": int(1 if rng.integers(2) else -1)})
    return out


# ---- directed graphs (in-degree graph Laplacian inputs) -------------------

def directed_powerlaw_graph(n, m, seed=3, gamma_in=2.1, gamma_out=2.7):
    """Edges (src, dst) of a directed graph with power-law degrees, no self
    loops, no repeated edges, exactly m >= n edges (Chung-Lu style).

    Node i has expected in-degree weight (r_in(i) + 1)^(-1/(gamma_in - 1)) and
    out-degree weight (r_out(i) + 1)^(-1/(gamma_out - 1)), r_in and r_out two
    independent random rankings.  Every node first receives one in-edge (as
    every page of a crawl was reached by a link), its source drawn from the
    out weights; the other edges draw their source from the out weights and
    their target from the in weights.  The exponents are the in-/out-degree
    exponents commonly reported for web graphs.
    """
    rng = np.random.default_rng(seed)
    w_in = (rng.permutation(n) + 1.0) ** (-1.0 / (gamma_in - 1.0))
    w_out = (rng.permutation(n) + 1.0) ** (-1.0 / (gamma_out - 1.0))
    w_in /= w_in.sum()
    w_out /= w_out.sum()
    dst0 = np.arange(n, dtype=np.int64)
    src0 = rng.choice(n, size=n, p=w_out)
    while np.any(src0 == dst0):  # no self loops
        bad = src0 == dst0
        src0[bad] = rng.choice(n, size=int(bad.sum()), p=w_out)
    first = src0 * n + dst0
    keys = np.zeros(0, dtype=np.int64)
    m_rest = m - n
    while keys.shape[0] < m_rest:
        k = int(1.2 * (m_rest - keys.shape[0])) + 1024
        src = rng.choice(n, size=k, p=w_out)
        dst = rng.choice(n, size=k, p=w_in)
        ok = src != dst
        new = src[ok].astype(np.int64) * n + dst[ok]
        keys = np.setdiff1d(np.unique(np.concatenate([keys, new])), first, assume_unique=True)
    keys = np.concatenate([first, keys[rng.permutation(keys.shape[0])[:m_rest]]])
    return (keys // n).astype(np.int64), (keys % n).astype(np.int64)


def graph_laplacian_csr(n, src, dst):
    """CSR (rowptr int64, col int32, val float64) of the in-degree Laplacian
    L = D_in - A, A[i, j] = 1 for an edge i -> j, D_in = diag(in-degrees) (the
    column sums of A), so every column of L sums to zero.  Columns ascending
    within a row; the diagonal is stored only where it is nonzero."""
    indeg = np.bincount(dst, minlength=n).astype(np.float64)
    diag = np.nonzero(indeg)[0]
    rows = np.concatenate([src, diag])
    cols = np.concatenate([dst, diag])
    vals = np.concatenate([-np.ones(src.shape[0]), indeg[diag]])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), vals


def unit_vector(n, seed=4):
    """A canonical unit vector e_i with i drawn from the seed (Sec. 6, Example 3 takes b = e_i)."""
    b = np.zeros(n)
    b[np.random.default_rng(seed).integers(n)] = 1.0
    return b
