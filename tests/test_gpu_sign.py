"""GPU parity of the sign-function path (PP_WILSON4D_Q2, Sec. 6 Example 2)
through the C ABI against the oracle (oracle/wilson.py, oracle/sign.py,
oracle/ritz.py).

A = Q^2 with Q = Gamma_5 D(m_w, mu) at the paper's m_w = -1.4, mu = 0.3
(non-Hermitian, complex Arnoldi), random Haar links.  Tolerances (relative
2-norm): one application of Q^2 1e-13 (FP64 and double-word: two stencil
applications of 17 terms each) and 2e-6 in FP32; q(A) v with complex
coefficients 1e-11 (FP64) / 5e-11 (double-word) for deg q <= 8; Ritz values
1e-9 relative (eigenvalues of the same 9 x 9 Hessenberg matrix, whose
entries carry the rounding of 9 Arnoldi steps); solves 1e-10 against the
dense sign function or a tolerance-1e-13 plain Arnoldi oracle (solve
tolerance 1e-12; double-word and mixed: 5e-10, as in the double-word Wilson
solves).
"""
import numpy as np
import pytest

import synth
from oracle import ritz, sign, wilson
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"f64": 0, "dw": 1, "mixed": 2}
MW, MU = -1.4, 0.3
SMALL = (2, 2, 2, 4)     # 384 complex unknowns: dense reference
MEDIUM = (4, 4, 2, 6)    # 2304 complex unknowns: 2 Wilson blocks of 128 sites ... 4.5 vector chunks


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


class Q2:
    def __init__(self, pp, dims, links, mu=MU, matrix=True):
        self.pp, self.dims = pp, tuple(dims)
        self.V = int(np.prod(dims))
        self.n = 12 * self.V
        self.links_d = dev(links.astype(np.complex64))
        self.h = pp.pp_create_stencil(pp.PP_WILSON4D_Q2, self.dims, [MW, mu], links=self.links_d,
                                      dtype=pp.PP_C128)
        self.Q = wilson.q_matrix(self.dims, links, MW, mu) if matrix else None

    def q2(self, v):
        return self.Q @ (self.Q @ v)

    def set(self, prec, side=0, orth=0, check_every=0):
        o = self.pp.pp_default_opts()
        o.precision = PREC[prec]
        o.side = side
        o.orth = orth
        o.check_every = check_every
        self.pp.pp_set_opts(self.h, o)

    def close(self):
        self.pp.pp_destroy(self.h)


_REF = {}


def reference(dims, seed_b):
    """sign(Q) b: dense for the small lattice, a tolerance-1e-13 plain CGS2 Arnoldi otherwise."""
    key = (dims, seed_b)
    if key not in _REF:
        links = synth.wilson_links(dims, 1)
        Q = wilson.q_matrix(dims, links, MW, MU)
        b = synth.spinor_field(dims, seed_b)
        if Q.shape[0] <= 1000:
            x = sign.sign_dense(Q.toarray()) @ b
        else:
            x, r = sign.sign_krylov(lambda v: Q @ v, b, orth="cgs2", m_max=1500, tol=1e-13, k_chk=8)
            assert r["converged"]
        _REF[key] = (b, x)
    return _REF[key]


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("dims", [SMALL, MEDIUM])
def test_q2_op_apply(dims, prec):
    pp = load()
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        pp.pp_build_poly(L.h, 0, interval_ab=(0.1, 50.0))
        L.set(prec)
        x = synth.spinor_field(dims, 11)
        yd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        pp.pp_op_apply(L.h, dev(x), yd)
        assert rel(host(yd), L.q2(x)) < (2e-6 if prec == "mixed" else 1e-13)
    finally:
        L.close()


def test_q2_free_field_symbol():
    # U = 1: Q^2 from the library against the Fourier closed form of the oracle
    pp = load()
    dims = (4, 2, 2, 6)
    L = Q2(pp, dims, synth.unit_links(dims))
    try:
        pp.pp_build_poly(L.h, 0, interval_ab=(0.1, 50.0))
        L.set("f64")
        x = synth.spinor_field(dims, 2)
        yd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        pp.pp_op_apply(L.h, dev(x), yd)
        sym = wilson.free_q_symbol(dims, MW, MU)
        assert rel(host(yd), wilson.free_spin_fun(dims, x, sym @ sym)) < 1e-13
    finally:
        L.close()


@pytest.mark.parametrize("harmonic", [False, True], ids=["ritz", "harmonic"])
@pytest.mark.parametrize("degree", [4, 8])
def test_complex_ritz_nodes(degree, harmonic):
    pp = load()
    dims = MEDIUM
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        L.set("f64")
        kind = pp.PP_HARMONIC_RITZ if harmonic else pp.PP_RITZ_LEJA
        pp.pp_build_poly(L.h, degree, kind)
        k, x, cap = pp.pp_get_poly_nodes(L.h)
        assert k == kind and len(x) == degree + 1
        xo, _ = ritz.ritz_poly(L.q2, L.n, degree, harmonic=harmonic, complex_=True, hermitian=False)
        # the same node set: the library keeps reverse Leja order
        assert np.max(np.abs(x - xo[::-1])) < 1e-9 * np.max(np.abs(xo))
        assert np.abs(np.imag(x)).max() > 1e-6  # genuinely complex, no conjugate pairs needed
    finally:
        L.close()


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("degree", [1, 2, 8])
def test_complex_poly_apply(degree, prec):
    pp = load()
    dims = MEDIUM
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        L.set(prec)
        pp.pp_build_poly(L.h, degree, pp.PP_RITZ_LEJA)
        _, x, _ = pp.pp_get_poly_nodes(L.h)
        v = synth.spinor_field(dims, 12)
        yd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        pp.pp_poly_apply(L.h, dev(v), yd)
        # q(A) v term by term at the library's own nodes (Newton sum, oracle)
        ref = ritz.newton_apply(L.q2, ritz.newton_coeffs(x), x, v)
        assert rel(host(yd), ref) < (1e-11 if prec == "f64" else 5e-11)
    finally:
        L.close()


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
@pytest.mark.parametrize("poly", [("plain", 0), ("ritz", 4), ("ritz", 8), ("harmonic", 8)])
@pytest.mark.parametrize("dims", [SMALL, MEDIUM])
def test_sign_solve(dims, poly, side, prec):
    pp = load()
    b, xs = reference(dims, 0)
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        L.set(prec, side=side)
        kind = {"plain": pp.PP_RITZ_LEJA, "ritz": pp.PP_RITZ_LEJA, "harmonic": pp.PP_HARMONIC_RITZ}[poly[0]]
        pp.pp_build_poly(L.h, poly[1], kind)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=1200, tol=1e-12)
        assert st.status == pp.PP_OK
        if prec == "mixed":  # kappa_pre estimated from H_m: FP32 for the tail of the run
            assert st.switch_iter < st.iters
        assert rel(host(xd), xs) < (1e-10 if prec == "f64" else 5e-10)
    finally:
        L.close()


def test_sign_matches_oracle_iterations():
    # the same method step for step: Ritz q of degree 8, left, CGS2, check every 2
    pp = load()
    dims = MEDIUM
    b, xs = reference(dims, 0)
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        o = pp.pp_default_opts()
        o.check_every = 2
        pp.pp_set_opts(L.h, o)
        pp.pp_build_poly(L.h, 8, pp.PP_RITZ_LEJA)
        _, x, _ = pp.pp_get_poly_nodes(L.h)
        a = ritz.newton_coeffs(x)
        qmv = lambda v: ritz.newton_apply(L.q2, a, x, v)
        xo, r = sign.sign_krylov(lambda v: L.Q @ v, b, orth="cgs2", m_max=400, tol=1e-12, k_chk=2,
                                 q=(len(a) - 1, qmv))
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=400, tol=1e-12)
        assert st.status == pp.PP_OK and r["converged"]
        assert st.iters == r["iters"]
        assert st.mvms == r["mvms"]
        assert rel(host(xd), xo) < 1e-11
    finally:
        L.close()


@pytest.mark.parametrize("f", [-1, 1], ids=["invsqrt", "sqrt"])
def test_q2_invsqrt_and_sqrt(f):
    # (Q^2)^{-1/2} b = sign(Q) Q^{-1} b and (Q^2)^{1/2} b = Q sign(Q) b (principal roots)
    pp = load()
    dims = SMALL
    links = synth.wilson_links(dims, 1)
    L = Q2(pp, dims, links)
    try:
        b = synth.spinor_field(dims, 3)
        Qd = L.Q.toarray()
        S = sign.sign_dense(Qd)
        ref = S @ np.linalg.solve(Qd, b) if f < 0 else Qd @ (S @ b)
        pp.pp_build_poly(L.h, 6, pp.PP_RITZ_LEJA)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, f, dev(b), xd, m_max=800, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), ref) < 1e-10
    finally:
        L.close()


def test_sign_chebyshev_q_on_complex_operator():
    # a real Chebyshev q on an interval around the real parts of the spectrum
    # is a valid preconditioner of the complex operator as well
    pp = load()
    dims = SMALL
    b, xs = reference(dims, 0)
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        lam = np.linalg.eigvals(L.Q.toarray()) ** 2
        pp.pp_build_poly(L.h, 6, pp.PP_CHEBYSHEV, interval_ab=(0.9 * lam.real.min(), 1.05 * lam.real.max()))
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=800, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), xs) < 1e-10
    finally:
        L.close()


def test_sign_free_field():
    pp = load()
    dims = (4, 2, 2, 6)
    L = Q2(pp, dims, synth.unit_links(dims))
    try:
        b = synth.spinor_field(dims, 7)
        sym = wilson.free_q_symbol(dims, MW, MU)
        S = np.empty_like(sym)
        for idx in np.ndindex(sym.shape[:4]):
            S[idx] = sign.sign_dense(sym[idx])
        ref = wilson.free_spin_fun(dims, b, S)
        pp.pp_build_poly(L.h, 4, pp.PP_RITZ_LEJA)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=800, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), ref) < 1e-10
    finally:
        L.close()


def test_sign_mu_zero_hermitian():
    # mu = 0: Q Hermitian, Q^2 HPD: the real-view Lanczos path; sign(Q) by eigh
    pp = load()
    dims = SMALL
    links = synth.wilson_links(dims, 1)
    L = Q2(pp, dims, links, mu=0.0)
    try:
        b = synth.spinor_field(dims, 4)
        lam, X = np.linalg.eigh(L.Q.toarray())
        ref = (X * np.sign(lam)) @ (X.conj().T @ b)
        pp.pp_build_poly(L.h, 6, pp.PP_RITZ_LEJA)
        _, x, _ = pp.pp_get_poly_nodes(L.h)
        assert not np.iscomplexobj(x)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=800, tol=1e-12)
        assert st.status == pp.PP_OK
        assert rel(host(xd), ref) < 1e-10
    finally:
        L.close()


def test_sign_zero_rhs_and_overlap():
    pp = load()
    dims = SMALL
    b, xs = reference(dims, 0)
    L = Q2(pp, dims, synth.wilson_links(dims, 1))
    try:
        pp.pp_build_poly(L.h, 4, pp.PP_RITZ_LEJA)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(np.zeros(L.n, dtype=np.complex128)), xd, m_max=50, tol=1e-12)
        assert st.status == pp.PP_OK and np.all(host(xd) == 0)
        # overlap operator D_ov b = b + rho Gamma_5 sign(Q) b from the library's sign(Q) b
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=800, tol=1e-12)
        rho = 0.9
        assert rel(sign.overlap_apply(b, host(xd), rho), sign.overlap_apply(b, xs, rho)) < 1e-10
    finally:
        L.close()


FULL = (16, 16, 16, 32)  # the lattice of the sign16x32 bench workload


@pytest.mark.parametrize("prec", ["dw", "mixed"])
def test_sign_free_field_full_size(prec):
    # U = 1 on 16^3 x 32 (n = 1,572,864 complex): the library's sign(Q) b with
    # the bench's q (Ritz, degree 31) against the per-momentum Fourier form
    pp = load()
    L = Q2(pp, FULL, synth.unit_links(FULL), matrix=False)
    try:
        b = synth.spinor_field(FULL, 7)
        sym = wilson.free_q_symbol(FULL, MW, MU)
        lam, X = np.linalg.eig(sym)
        S = X @ (np.sign(lam.real)[..., None] * np.linalg.inv(X))
        ref = wilson.free_spin_fun(FULL, b, S)
        L.set(prec, check_every=2)
        pp.pp_build_poly(L.h, 31, pp.PP_RITZ_LEJA)
        xd = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        st = pp.pp_apply(L.h, pp.PP_SIGN, dev(b), xd, m_max=300, tol=1e-11)
        assert st.status == pp.PP_OK
        assert rel(host(xd), ref) < 1e-9
    finally:
        L.close()


def test_sign_identities_full_size():
    # random SU(3) links on 16^3 x 32: sign(Q)^2 b = b and
    # (Q^2)^{-1/2} (Q^2)^{1/2} b = b through the library alone
    pp = load()
    L = Q2(pp, FULL, synth.wilson_links(FULL, 1), matrix=False)
    try:
        L.set("dw", check_every=2)
        pp.pp_build_poly(L.h, 31, pp.PP_RITZ_LEJA)
        b = dev(synth.spinor_field(FULL, 0))
        x1 = torch.empty(L.n, dtype=torch.complex128, device="cuda")
        x2 = torch.empty_like(x1)
        assert pp.pp_apply(L.h, pp.PP_SIGN, b, x1, m_max=300, tol=1e-12).status == pp.PP_OK
        assert pp.pp_apply(L.h, pp.PP_SIGN, x1, x2, m_max=300, tol=1e-12).status == pp.PP_OK
        assert rel(host(x2), host(b)) < 1e-10
        assert pp.pp_apply(L.h, pp.PP_SQRT, b, x1, m_max=300, tol=1e-12).status == pp.PP_OK
        assert pp.pp_apply(L.h, pp.PP_INVSQRT, x1, x2, m_max=300, tol=1e-12).status == pp.PP_OK
        assert rel(host(x2), host(b)) < 1e-10
    finally:
        L.close()
