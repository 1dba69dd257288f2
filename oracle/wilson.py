"""Wilson-type lattice operator D and A = D^H D, FP64 / complex128 (test infrastructure only).

Not in the paper as such: Sec. 6, Example 2 applies the method to the
overlap operator, whose kernel is built from a Wilson-Dirac operator on a
QCD configuration that is not available here.  The stand-in is the Hermitian
positive definite A = D^H D of a Wilson-type operator on a periodic 4D
lattice with random SU(3) links:

    (D psi)(x) = (4 + m0) psi(x)
                 - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ],

mu = 0..3 the lattice directions x, y, z, t with gamma_1..gamma_4, periodic
boundaries in all four directions, m0 the mass shift.  The gamma matrices are
the Euclidean chiral representation (Hermitian, gamma_5 = diag(1,1,-1,-1)):

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1,2,3),  gamma_4 = [[0, I], [I, 0]].

Vector layout: 12 complex entries per site, index s*12 + spin*3 + colour,
site s = ((t Lz + z) Ly + y) Lx + x.  Links: array [s, mu, a, b] = U_mu(s)_{ab}.

Closed form for the free field U = 1 (momenta p_mu = 2 pi k_mu / L_mu):
A(p) = (m0 + sum_mu (1 - cos p_mu))^2 + sum_mu sin^2 p_mu times the 12 x 12
identity, so f(A) b is a spectral multiplier after a 4D FFT.
"""
import numpy as np
import scipy.sparse as sp

_SIGMA = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
          np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          np.array([[1, 0], [0, -1]], dtype=np.complex128)]


def gammas():
    """(gamma_1, gamma_2, gamma_3, gamma_4, gamma_5) of the chiral representation."""
    Z = np.zeros((2, 2), dtype=np.complex128)
    I2 = np.eye(2, dtype=np.complex128)
    g = [np.block([[Z, -1j * s], [1j * s, Z]]) for s in _SIGMA]
    g.append(np.block([[Z, I2], [I2, Z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g + [g5]


def neighbours(dims, mu, sign):
    """Site index of x + sign * e_mu (periodic) for every site x."""
    dims = tuple(int(L) for L in dims)
    V = int(np.prod(dims))
    s = np.arange(V)
    coords = []
    rem = s.copy()
    for L in dims:
        coords.append(rem % L)
        rem //= L
    coords[mu] = (coords[mu] + sign) % dims[mu]
    idx = np.zeros(V, dtype=np.int64)
    stride = 1
    for d, L in enumerate(dims):
        idx += coords[d] * stride
        stride *= L
    return idx


def dirac_matrix(dims, links, m0, mu_c=0.0):
    """Sparse complex128 matrix of D (12 V x 12 V).

    mu_c: chemical potential (Sec. 6, Example 2): the hop to x + t carries the
    factor e^{mu_c}, the hop to x - t the factor e^{-mu_c} (t = direction 3,
    gamma_4); mu_c = 0 is the operator above.
    """
    dims = tuple(int(L) for L in dims)
    V = int(np.prod(dims))
    U = np.asarray(links).astype(np.complex128).reshape(V, 4, 3, 3)
    g = gammas()
    I4 = np.eye(4, dtype=np.complex128)
    rows, cols, vals = [], [], []
    base = np.arange(12)
    for mu in range(4):
        for sign in (+1, -1):
            nb = neighbours(dims, mu, sign)
            chem = np.exp(sign * mu_c) if mu == 3 else 1.0
            if sign > 0:
                spin = -0.5 * chem * (I4 - g[mu])
                col_mats = U[:, mu]                                  # U_mu(x)
            else:
                spin = -0.5 * chem * (I4 + g[mu])
                col_mats = np.conj(np.transpose(U[nb, mu], (0, 2, 1)))  # U_mu(x - mu)^H
            # block[s] = kron(spin, colour[s]) : 12 x 12
            blocks = np.einsum("ij,sab->siajb", spin, col_mats).reshape(V, 12, 12)
            r = (np.arange(V)[:, None, None] * 12 + base[None, :, None]) + 0 * base[None, None, :]
            c = (nb[:, None, None] * 12 + base[None, None, :]) + 0 * base[None, :, None]
            keep = blocks != 0
            rows.append(r[keep])
            cols.append(c[keep])
            vals.append(blocks[keep])
    rows.append(np.arange(12 * V))
    cols.append(np.arange(12 * V))
    vals.append(np.full(12 * V, 4.0 + m0, dtype=np.complex128))
    D = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(12 * V, 12 * V))
    return D.tocsr()


def q_matrix(dims, links, m_w, mu_c):
    """Q = Gamma_5 D(m_w, mu_c) (Sec. 6, Example 2), sparse; Gamma_5 = diag(1, 1, -1, -1) on spin."""
    D = dirac_matrix(dims, links, m_w, mu_c)
    V = D.shape[0] // 12
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
    return (sp.diags(g5) @ D).tocsr()


def dhd_matrix(dims, links, m0):
    """A = D^H D as a sparse matrix."""
    D = dirac_matrix(dims, links, m0)
    return (D.conj().T @ D).tocsr()


def free_eigs(dims, m0):
    """lambda(p) of A for U = 1 on the FFT grid, shape (Lt, Lz, Ly, Lx)."""
    dims = tuple(int(L) for L in dims)
    shape = tuple(reversed(dims))
    M = np.full(shape, float(m0))
    S2 = np.zeros(shape)
    for mu, L in enumerate(dims):
        p = 2.0 * np.pi * np.arange(L) / L
        sh = [1, 1, 1, 1]
        sh[3 - mu] = L
        M = M + (1.0 - np.cos(p)).reshape(sh)
        S2 = S2 + (np.sin(p) ** 2).reshape(sh)
    return M * M + S2


def free_field_fun(dims, b, power, m0):
    """f(A) b = A^power b for the free field U = 1 by the 4D FFT closed form."""
    dims = tuple(int(L) for L in dims)
    X = np.asarray(b, dtype=np.complex128).reshape(tuple(reversed(dims)) + (12,))
    F = np.fft.fftn(X, axes=(0, 1, 2, 3))
    F = F * np.power(free_eigs(dims, m0), power)[..., None]
    return np.fft.ifftn(F, axes=(0, 1, 2, 3)).reshape(-1)


def gauge_transform(dims, links, G):
    """U'_mu(x) = G(x) U_mu(x) G(x + mu)^H for G of shape (V, 3, 3)."""
    V = int(np.prod(dims))
    U = np.asarray(links).astype(np.complex128).reshape(V, 4, 3, 3)
    out = np.empty_like(U)
    for mu in range(4):
        nb = neighbours(dims, mu, +1)
        out[:, mu] = G @ U[:, mu] @ np.conj(np.transpose(G[nb], (0, 2, 1)))
    return out


def gauge_apply(G, psi):
    """(G psi)(x) = G(x) psi(x) on the colour index of every spin component."""
    V = G.shape[0]
    P = np.asarray(psi).reshape(V, 4, 3)
    return np.einsum("sab,sjb->sja", G, P).reshape(-1)


def gamma5_apply(psi):
    """gamma_5 = diag(1, 1, -1, -1) on the spin index."""
    P = np.asarray(psi).reshape(-1, 4, 3).copy()
    P[:, 2:] *= -1.0
    return P.reshape(-1)


def free_q_symbol(dims, m_w, mu_c):
    """Q(p) = gamma_5 D(p) for U = 1: the 4 x 4 spin matrix of Q at every FFT
    momentum, shape (Lt, Lz, Ly, Lx, 4, 4).

    A plane wave e^{i p.x} u is an eigenvector of the hops, with e^{+-i p_mu}
    for the hop to x +- mu and, in direction t, the extra factors e^{+-mu_c}:
    with p~_t = p_t - i mu_c (p~ = p otherwise),
        D(p) = (m_w + sum_mu (1 - cos p~_mu)) I + i sum_mu gamma_mu sin p~_mu.
    """
    dims = tuple(int(L) for L in dims)
    shape = tuple(reversed(dims))
    g = gammas()
    M = np.full(shape, complex(m_w))
    S = [None] * 4
    for mu, L in enumerate(dims):
        p = (2.0 * np.pi * np.arange(L) / L).astype(np.complex128)
        if mu == 3:
            p = p - 1j * mu_c
        sh = [1, 1, 1, 1]
        sh[3 - mu] = L
        M = M + (1.0 - np.cos(p)).reshape(sh)
        S[mu] = np.broadcast_to(np.sin(p).reshape(sh), shape)
    D = M[..., None, None] * np.eye(4) + 1j * sum(S[mu][..., None, None] * g[mu] for mu in range(4))
    return g[4] @ D


def free_spin_fun(dims, b, mats):
    """(F b) for a per-momentum 4 x 4 spin matrix field mats (identity on colour) by the 4D FFT."""
    dims = tuple(int(L) for L in dims)
    X = np.asarray(b, dtype=np.complex128).reshape(tuple(reversed(dims)) + (4, 3))
    F = np.fft.fftn(X, axes=(0, 1, 2, 3))
    F = np.einsum("...ij,...jc->...ic", mats, F)
    return np.fft.ifftn(F, axes=(0, 1, 2, 3)).reshape(-1)
