"""Pins of the oracle's sign-function path (oracle/sign.py, the chemical
potential and Q = Gamma_5 D of oracle/wilson.py, unpaired complex Leja
nodes of oracle/ritz.py) against what the mathematics fixes: the free-field
Fourier symbol of Q with the shifted momentum p_t - i mu, gamma_5-hermiticity
D(mu)^H = Gamma_5 D(-mu) Gamma_5, sign(Q)^2 = I and [sign(Q), Q] = 0, the
Hermitian case by eigh, the Ginsparg-Wilson relation of the overlap
operator, and the Leja property by brute force (Sec. 5.2, Sec. 6 Example 2)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import krylov, ritz, sign, wilson

MW, MU = -1.4, 0.3  # the shift and chemical potential of Sec. 6, Example 2


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def g5_vec(V):
    return np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)


@pytest.mark.parametrize("dims", [(4, 3, 2, 6), (2, 2, 4, 3)])
@pytest.mark.parametrize("mu", [0.0, MU, -0.7])
def test_free_q_symbol_matches_sparse(dims, mu):
    Q = wilson.q_matrix(dims, synth.unit_links(dims), MW, mu)
    b = synth.spinor_field(dims, 3)
    ref = wilson.free_spin_fun(dims, b, wilson.free_q_symbol(dims, MW, mu))
    assert rel(Q @ b, ref) < 1e-13


def test_chemical_potential_adjoint_relation():
    dims = (2, 3, 2, 4)
    U = synth.wilson_links(dims, seed=5)
    V = int(np.prod(dims))
    G5 = np.diag(g5_vec(V))
    Dp = wilson.dirac_matrix(dims, U, MW, MU).toarray()
    Dm = wilson.dirac_matrix(dims, U, MW, -MU).toarray()
    assert np.abs(Dp.conj().T - G5 @ Dm @ G5).max() < 1e-14
    Q0 = wilson.q_matrix(dims, U, MW, 0.0).toarray()
    assert np.abs(Q0 - Q0.conj().T).max() < 1e-14          # mu = 0: Q Hermitian
    Qp = wilson.q_matrix(dims, U, MW, MU).toarray()
    assert np.abs(Qp - Qp.conj().T).max() > 0.1              # mu != 0: not Hermitian
    Qm = wilson.q_matrix(dims, U, MW, -MU).toarray()
    assert np.abs(Qp.conj().T - Qm).max() < 1e-14            # Q(mu)^H = Q(-mu)


def test_sign_dense_definition():
    dims = (2, 2, 2, 2)
    U = synth.wilson_links(dims, seed=2)
    Q = wilson.q_matrix(dims, U, MW, MU).toarray()
    S = sign.sign_dense(Q)
    I = np.eye(Q.shape[0])
    assert np.abs(S @ S - I).max() < 1e-10
    assert np.abs(S @ Q - Q @ S).max() < 1e-10
    # Hermitian Q (mu = 0): the sign of the eigenvalues of eigh
    Q0 = wilson.q_matrix(dims, U, MW, 0.0).toarray()
    lam, X = np.linalg.eigh(Q0)
    assert np.abs(sign.sign_dense(Q0) - (X * np.sign(lam)) @ X.conj().T).max() < 1e-10


def test_sign_free_field_closed_form():
    dims = (4, 2, 2, 4)
    Q = wilson.q_matrix(dims, synth.unit_links(dims), MW, MU)
    b = synth.spinor_field(dims, 7)
    sym = wilson.free_q_symbol(dims, MW, MU)
    S = np.empty_like(sym)
    for idx in np.ndindex(sym.shape[:4]):
        S[idx] = sign.sign_dense(sym[idx])
    ref = wilson.free_spin_fun(dims, b, S)
    x, r = sign.sign_krylov(lambda v: Q @ v, b, orth="cgs2", m_max=400, tol=1e-13, k_chk=4)
    assert r["converged"]
    assert rel(x, ref) < 1e-10


@pytest.mark.parametrize("harmonic", [False, True])
def test_sign_krylov_ritz_preconditioned(harmonic):
    dims = (2, 2, 2, 4)
    U = synth.wilson_links(dims, seed=1)
    Q = wilson.q_matrix(dims, U, MW, MU)
    n = Q.shape[0]
    b = synth.spinor_field(dims, 0)
    ref = sign.sign_dense(Q.toarray()) @ b

    def Q2(v):
        return Q @ (Q @ v)

    x_nodes, a = ritz.ritz_poly(Q2, n, 6, harmonic=harmonic, complex_=True, hermitian=False)
    assert len(x_nodes) == 7 and np.abs(np.imag(x_nodes)).max() > 0
    # interpolation: q(theta_i) = theta_i^{-1/2} at every Ritz value
    vals = ritz.newton_eval(a, x_nodes, x_nodes)
    assert np.abs(vals - x_nodes ** -0.5).max() < 1e-9 * np.abs(x_nodes ** -0.5).max()
    # Sec. 4: positivity of q at the Ritz values (all in the right half-plane here)
    assert np.all(np.real(x_nodes) > 0) and np.all(np.real(vals) > 0)
    qmv = lambda v: ritz.newton_apply(Q2, a, x_nodes, v)
    x, r = sign.sign_krylov(lambda v: Q @ v, b, orth="cgs2", m_max=200, tol=1e-12, k_chk=2,
                            q=(len(a) - 1, qmv))
    assert r["converged"]
    assert rel(x, ref) < 1e-9
    x0, r0 = sign.sign_krylov(lambda v: Q @ v, b, orth="cgs2", m_max=400, tol=1e-12, k_chk=2)
    assert r["iters"] < r0["iters"]


def test_overlap_ginsparg_wilson():
    dims = (2, 2, 2, 2)
    U = synth.wilson_links(dims, seed=3)
    Q = wilson.q_matrix(dims, U, MW, MU).toarray()
    S = sign.sign_dense(Q)
    n = Q.shape[0]
    I = np.eye(n, dtype=np.complex128)
    Dov = np.stack([sign.overlap_apply(I[:, k], S[:, k], 1.0) for k in range(n)], axis=1)
    G5 = np.diag(g5_vec(n // 12))
    # rho = 1: gamma_5 D + D gamma_5 = D gamma_5 D (needs only sign(Q)^2 = I)
    assert np.abs(G5 @ Dov + Dov @ G5 - Dov @ G5 @ Dov).max() < 1e-10
    assert np.abs(Dov - (I + G5 @ S)).max() < 1e-14


def test_leja_unpaired_brute_force():
    rng = np.random.default_rng(11)
    z = rng.standard_normal(7) + 1j * rng.standard_normal(7) + 3.0
    x = ritz.leja_order(z, pairs=False)
    assert sorted(map(complex, x), key=lambda c: (c.real, c.imag)) == \
        sorted(map(complex, z), key=lambda c: (c.real, c.imag))
    assert abs(x[0]) == np.abs(z).max()
    for i in range(1, len(x)):
        rest = x[i:]
        score = [np.prod(np.abs(r - x[:i])) for r in rest]
        assert np.prod(np.abs(x[i] - x[:i])) == max(score)
    # pairs=True on the same set (not conjugation-closed) would add conjugates
    y = ritz.leja_order(np.concatenate([z, z.conj()]), pairs=True)
    for i in range(0, len(y), 2):
        assert y[i + 1] == np.conj(y[i])


def test_mutation_is_caught():
    # a chemical potential on the wrong hop (e^{-mu} forward) breaks the free-field symbol
    dims = (2, 2, 2, 4)
    b = synth.spinor_field(dims, 1)
    Qwrong = wilson.q_matrix(dims, synth.unit_links(dims), MW, -MU)
    ref = wilson.free_spin_fun(dims, b, wilson.free_q_symbol(dims, MW, MU))
    assert rel(Qwrong @ b, ref) > 1e-3
