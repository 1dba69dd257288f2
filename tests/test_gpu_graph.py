"""GPU parity of Example 3's problem class through the C ABI: L^{1/2} b for
the in-degree Laplacian L of a directed graph (non-Hermitian CSR, singular
with a semi-simple zero eigenvalue), computed as L^{-1/2}(L b) (Sec. 4) with
Arnoldi + CGS2 and q interpolating at Ritz or harmonic Ritz values
(Sec. 5.2).  The reference is the oracle's plain Arnoldi at tolerance 1e-13
(the paper's reference for this example; it agrees with the dense Schur
root to 2e-14 on this graph); the library's solves run at 1e-11 and must
land within 1e-7 of it, Example 3's target, in FP64, double-word and mixed
precision.  (The degree-15 Ritz interpolant is large between its nodes and
amplifies the rounding of the operator chain: FP64 lands at 2e-9, and the
double-word path meets the target because its CSR step computes in FP64.)
Ritz interpolants need not be positive on the whole spectrum (Sec. 5.2
argues it at the Ritz values only): the tests check positivity against the
dense eigenvalues and, where it fails, that the library returns the root
the method then defines."""
import functools

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import krylov, ritz
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"f64": 0, "dw": 1, "mixed": 2}
N, M = 1500, 12000
TOL = 1e-7  # Example 3's target, for every precision
# (degree, kind) whose q is positive on the whole spectrum of this graph
# (checked against the dense eigenvalues in the test), and ones where it is
# not: Sec. 5.2 can only argue positivity at the Ritz values
POSITIVE = [(0, "ritz"), (0, "harmonic"), (3, "harmonic"), (7, "ritz"), (7, "harmonic"), (15, "ritz"),
            (15, "harmonic")]
NEGATIVE = [(1, "ritz"), (1, "harmonic"), (3, "ritz")]


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@functools.lru_cache(maxsize=None)
def graph():
    src, dst = synth.directed_powerlaw_graph(N, M, seed=5)
    return synth.graph_laplacian_csr(N, src, dst)


def matrix():
    rp, col, val = graph()
    return sp.csr_matrix((val, col, rp), shape=(N, N))


@functools.lru_cache(maxsize=None)
def eig():
    lam, V = np.linalg.eig(matrix().toarray())
    return lam, V


def rhs(bseed):
    return synth.unit_vector(N, bseed) if bseed >= 0 else synth.rhs(N, -bseed)


@functools.lru_cache(maxsize=None)
def reference(bseed):
    b = rhs(bseed)
    r = krylov.pp_arnoldi(matrix().dot, b, 0.5, m_max=N, tol=1e-13, k_chk=8, orth="cgs2")
    assert r["converged"]
    return b, r["x"]


def handle(pp, prec):
    rp, col, val = graph()
    keep = [dev(rp), dev(col), dev(val)]
    h = pp.pp_create_csr(N, *keep, is_hermitian=False)
    o = pp.pp_default_opts()
    o.precision = PREC[prec]
    pp.pp_set_opts(h, o)
    return h, keep


def kind_of(pp, kind):
    return {"ritz": pp.PP_RITZ_LEJA, "harmonic": pp.PP_HARMONIC_RITZ}[kind]


def q_on_spectrum(pp, h):
    _, x, _ = pp.pp_get_poly_nodes(h)
    a, _, _ = pp.pp_get_poly(h)
    lam, _ = eig()
    return x, a, ritz.newton_eval(a, x, lam)


def solve_and_compare(pp, h, b, xref, degree, prec):
    # stopping checks every 32/d iterations, Example 3's cadence
    o = pp.pp_default_opts()
    o.precision = PREC[prec]
    o.check_every = max(1, 32 // (degree + 1))
    pp.pp_set_opts(h, o)
    xd = torch.empty(N, dtype=torch.float64, device="cuda")
    st = pp.pp_apply(h, pp.PP_SQRT, dev(b), xd, m_max=800, tol=1e-11)
    assert st.status == pp.PP_OK
    assert rel(host(xd), xref) < TOL
    # with a preconditioner, the 64/d cadence of Example 1 gives the same answer.
    # (Not for plain Arnoldi, degree 0: on this singular L its iterates reach
    # 1e-13 and then drift away, rounding feeding the null space of L into the
    # basis -- after about 200 steps in FP64, 170 in double-word -- and checks
    # 64 steps apart let the double-word run pass that point before its
    # estimate falls below 1e-11.)
    if degree > 0:
        o.check_every = 0
        pp.pp_set_opts(h, o)
        st = pp.pp_apply(h, pp.PP_SQRT, dev(b), xd, m_max=800, tol=1e-11)
        assert st.status == pp.PP_OK and rel(host(xd), xref) < TOL


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("dk", POSITIVE, ids=lambda t: f"{t[0]}{t[1]}")
@pytest.mark.parametrize("bseed", [4, 9], ids=["e_i", "e_j"])
def test_graph_laplacian_sqrt(bseed, dk, prec):
    # Example 3's setting, b a canonical unit vector, q positive on the spectrum
    degree, kind = dk
    pp = load()
    h, keep = handle(pp, prec)
    try:
        pp.pp_build_poly(h, degree, kind_of(pp, kind))
        x, a, q = q_on_spectrum(pp, h)
        assert np.all(np.real(x) > 0)
        assert q.real.min() > 0  # the method's premise holds for this q on this graph
        b, xref = reference(bseed)
        solve_and_compare(pp, h, b, xref, degree, prec)
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("dk", [t for t in POSITIVE if t[0] <= 7], ids=lambda t: f"{t[0]}{t[1]}")
def test_graph_laplacian_sqrt_random_b(dk, prec):
    # b ~ N(0,1) excites every eigenvector (at degree 15 the interpolant is so
    # large between the Ritz values that the oracle's own runs lose accuracy)
    degree, kind = dk
    pp = load()
    h, keep = handle(pp, prec)
    try:
        pp.pp_build_poly(h, degree, kind_of(pp, kind))
        _, _, q = q_on_spectrum(pp, h)
        assert q.real.min() > 0
        b, xref = reference(-1)
        solve_and_compare(pp, h, b, xref, degree, prec)
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("dk", NEGATIVE, ids=lambda t: f"{t[0]}{t[1]}")
def test_graph_nonpositive_q_follows_the_method(dk, prec):
    # q(lambda) < 0 for some eigenvalues: the method then converges to
    # q(A) (A q(A)^2)^{-1/2} A b, not to the principal root (Sec. 5.2 argues
    # positivity at the Ritz values only).  The library must agree with the
    # oracle's Algorithm 1 run with the library's own q.
    degree, kind = dk
    pp = load()
    h, keep = handle(pp, prec)
    try:
        pp.pp_build_poly(h, degree, kind_of(pp, kind))
        x, a, q = q_on_spectrum(pp, h)
        assert q.real.min() < 0
        b = rhs(-1)
        L = matrix()
        r = krylov.pp_arnoldi(L.dot, b, 0.5, q=(degree, lambda v: ritz.newton_apply(L.dot, a, x, v)),
                              m_max=800, tol=1e-11, k_chk=max(1, 64 // (degree + 1)), orth="cgs2")
        assert r["converged"]
        xd = torch.empty(N, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, pp.PP_SQRT, dev(b), xd, m_max=800, tol=1e-11)
        assert st.status == pp.PP_OK
        assert rel(host(xd), r["x"]) < 1e-6
        _, xref = reference(-1)
        assert rel(host(xd), xref) > 1e-3
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("degree", [3, 15])
def test_graph_ritz_nodes_match_oracle(degree):
    # the node run (CGS2 Arnoldi on L from the SplitMix64 start, Francis QR of
    # H_d) against the oracle's on the same start vector
    pp = load()
    h, keep = handle(pp, "f64")
    try:
        pp.pp_build_poly(h, degree, pp.PP_RITZ_LEJA)
        _, x, _ = pp.pp_get_poly_nodes(h)
        xo, _ = ritz.ritz_poly(matrix().dot, N, degree, hermitian=False)
        assert len(x) == len(xo)
        tol = 1e-8 * np.abs(xo).max()
        assert max(np.abs(np.asarray(xo) - z).min() for z in np.atleast_1d(x)) < tol
    finally:
        pp.pp_destroy(h)


def test_graph_sqrt_identity():
    # (L^{1/2})^2 b = L b through the library alone (b = e_i)
    pp = load()
    h, keep = handle(pp, "dw")
    try:
        pp.pp_build_poly(h, 7, pp.PP_RITZ_LEJA)
        b = synth.unit_vector(N, 3)
        x1 = torch.empty(N, dtype=torch.float64, device="cuda")
        x2 = torch.empty(N, dtype=torch.float64, device="cuda")
        lb = torch.empty(N, dtype=torch.float64, device="cuda")
        assert pp.pp_apply(h, pp.PP_SQRT, dev(b), x1, m_max=800, tol=1e-12).status == pp.PP_OK
        assert pp.pp_apply(h, pp.PP_SQRT, x1, x2, m_max=800, tol=1e-12).status == pp.PP_OK
        pp.pp_op_apply(h, dev(b), lb)
        assert rel(host(x2), host(lb)) < TOL
    finally:
        pp.pp_destroy(h)
