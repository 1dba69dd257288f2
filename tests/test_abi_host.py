"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, and its host-side construction (Chebyshev polynomial, quadrature
rule of the small solve, argument validation) agrees with the oracle."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import chebyshev as cheb, lsq, operators as ops, ritz
from tests.libpp import load

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(pp_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    pp = load()
    names = declared_functions()
    assert "pp_apply" in names and "pp_build_poly" in names and "pp_create_csr" in names
    out = subprocess.run(["nm", "-D", "--defined-only", pp.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(pp.lib(), n)
    assert set(names) == set(pp.SYMBOLS)  # the binding covers the whole header


def test_version_and_strerror():
    pp = load()
    assert pp.pp_version() >= 100
    assert pp.pp_strerror(pp.PP_ERR_NONPRIMARY) == "PP_ERR_NONPRIMARY"
    assert pp.pp_strerror(-99) == "PP_ERR_UNKNOWN"


@pytest.mark.parametrize("dims", [(50, 50), (64, 64), (33, 17)])
@pytest.mark.parametrize("degree", [0, 1, 8, 16, 31])
def test_build_poly_matches_oracle_2d(dims, degree):
    pp = load()
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    try:
        pp.pp_build_poly(h, degree)
        c, ab, img = pp.pp_get_poly(h)
        a, b = ops.laplace_interval(dims)
        assert np.allclose(ab, (a, b), rtol=1e-14)
        ref = cheb.interp_coeffs(a, b, degree + 1)
        assert np.max(np.abs(c - ref)) <= 1e-13 * np.max(np.abs(ref))
        lo, hi = cheb.image_interval(ref, a, b, npts=20001)
        assert abs(img[0] - lo) < 1e-9 and abs(img[1] - hi) < 1e-9
    finally:
        pp.pp_destroy(h)


def test_build_poly_convdiff_interval():
    pp = load()
    dims = (40, 30, 20)
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    try:
        pp.pp_build_poly(h, 4)
        c, ab, img = pp.pp_get_poly(h)
        assert np.allclose(ab, ops.convdiff_interval(dims, 0.5), rtol=1e-14)
        assert np.allclose(c, cheb.interp_coeffs(ab[0], ab[1], 5), rtol=1e-13, atol=1e-15)
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("kind,herm", [(0, True), (2, False)])
def test_quadrature_rule_accuracy(kind, herm):
    # sum_k w_k / (s_k + z) = z^{-1/2} on the (widened) image interval; complex z with
    # |arg z| <= pi/3 for the non-Hermitian case
    pp = load()
    h = (pp.pp_create_stencil(pp.PP_LAPLACE2D5, (64, 64)) if herm else
         pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (32, 32, 32), [0.5]))
    try:
        pp.pp_build_poly(h, 8)
        _, _, img = pp.pp_get_poly(h)
        s, w = pp.pp_get_quadrature(h)
        assert np.all(s > 0) and np.all(w > 0) and len(s) < 600
        z = np.geomspace(img[0] * 1e-3, img[1] * 1e3, 3001)
        if not herm:
            z = (z[:, None] * np.exp(1j * np.linspace(-np.pi / 3, np.pi / 3, 7))[None, :]).ravel()
        approx = (w[None, :] / (s[None, :] + z[:, None])).sum(1)
        assert np.max(np.abs(approx * np.sqrt(z) - 1)) < 1e-13
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("nodes", [
    [0.8, 1.5 + 0.7j, 1.5 - 0.7j, 3.0 + 1.2j, 3.0 - 1.2j, 5.0, 2.2],
    [0.8, 2.0 + 2.5j, 2.0 - 2.5j, 5.0, 2.2],
], ids=["pairs7", "wide_pair"])
def test_quadrature_rule_on_wide_sectors(nodes):
    # complex q nodes widen the sector the small solve's rule must cover
    # (1.5 |arg| of the widest node, at most 0.45 pi): the rule still gives
    # z^{-1/2} to 1e-13 over the widened image interval and that sector
    pp = load()
    z = np.array(nodes)
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (5, 4, 3), [0.5])
    try:
        pp.pp_set_poly_nodes(h, z, interval_ab=(0.2, 7.0))
        _, _, img = pp.pp_get_poly(h)
        s, w = pp.pp_get_quadrature(h)
        theta = max(np.pi / 3, min(0.45 * np.pi, 1.5 * np.max(np.abs(np.angle(z)))))
        assert np.all(s > 0) and np.all(w > 0) and len(s) < 600
        r = np.geomspace(img[0] * 1e-3, img[1] * 1e3, 2001)
        zz = (r[:, None] * np.exp(1j * np.linspace(-theta, theta, 9))[None, :]).ravel()
        approx = (w[None, :] / (s[None, :] + zz[:, None])).sum(1)
        assert np.max(np.abs(approx * np.sqrt(zz) - 1)) < 1e-13
    finally:
        pp.pp_destroy(h)


def test_quadrature_rule_is_compact():
    # the sinh-substituted rule needs far fewer nodes than the plain trapezoid
    # rule in log t at the same accuracy: on the 128^3 convection-diffusion
    # image (widened by 10^3) the plain rule takes about 450 nodes
    pp = load()
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (128, 128, 128), [0.5])
    try:
        pp.pp_build_poly(h, 16)
        s, w = pp.pp_get_quadrature(h)
        assert len(s) < 250
    finally:
        pp.pp_destroy(h)


def test_option_ranges():
    pp = load()
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, (8, 8))
    try:
        for field, good, bad in (("orth", (0, 1, 2, 3), (-1, 4)), ("halo", (0, 1), (2, -1)),
                                 ("clenshaw", (0, 1), (2,)), ("two_pass", (0, 1), (2,))):
            for v in good:
                o = pp.pp_default_opts()
                setattr(o, field, v)
                pp.pp_set_opts(h, o)
            for v in bad:
                o = pp.pp_default_opts()
                setattr(o, field, v)
                with pytest.raises(pp.PPError) as e:
                    pp.pp_set_opts(h, o)
                assert e.value.status == pp.PP_ERR_INVALID_ARG, (field, v)
    finally:
        pp.pp_destroy(h)


def test_argument_validation():
    pp = load()
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_LAPLACE3D7, (0, 4, 4))
    assert e.value.status == pp.PP_ERR_INVALID_ARG
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (4, 4, 4))  # needs c*h
    assert e.value.status == pp.PP_ERR_INVALID_ARG
    # Wilson: complex128 vectors, links and a finite mass required (host checks only)
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_WILSON4D_DHD, (4, 4, 4, 4), [0.1], links=64)
    assert e.value.status == pp.PP_ERR_UNSUPPORTED
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_WILSON4D_DHD, (4, 4, 4, 4), [0.1], dtype=pp.PP_C128)
    assert e.value.status == pp.PP_ERR_INVALID_ARG
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_WILSON4D_DHD, (4, 0, 4, 4), [0.1], links=64, dtype=pp.PP_C128)
    assert e.value.status == pp.PP_ERR_INVALID_ARG
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_WILSON4D_DHD, (4, 4, 4, 4), [float("nan")], links=64, dtype=pp.PP_C128)
    assert e.value.status == pp.PP_ERR_INVALID_ARG
    hw = pp.pp_create_stencil(pp.PP_WILSON4D_DHD, (4, 4, 4, 4), [0.1], links=64, dtype=pp.PP_C128)
    pp.pp_destroy(hw)
    # Wilson Q^2 (sign function): params = {m_w, mu}, mu finite
    with pytest.raises(pp.PPError) as e:
        pp.pp_create_stencil(pp.PP_WILSON4D_Q2, (4, 4, 4, 4), [-1.4, float("nan")], links=64, dtype=pp.PP_C128)
    assert e.value.status == pp.PP_ERR_INVALID_ARG
    hq = pp.pp_create_stencil(pp.PP_WILSON4D_Q2, (4, 4, 4, 4), [-1.4, 0.3], links=64, dtype=pp.PP_C128)
    try:
        # least squares on a contour of a complex operator: any point set (host work only)
        t = 2.0 * np.pi * np.arange(200) / 200
        z = (5.0 + 0.6j) + 4.0 * np.cos(t) + 1.2j * np.sin(t)
        pp.pp_set_poly_lsq(hq, 4, z)
        kind, x, _ = pp.pp_get_poly_nodes(hq)
        assert kind == pp.PP_LSQ_CONTOUR and len(x) == 5 and np.any(np.abs(np.imag(x)) > 0)
        assert all(np.min(np.abs(z - v)) < 1e-12 for v in x)  # Leja points of the contour
        with pytest.raises(pp.PPError) as e:  # Chebyshev needs the interval
            pp.pp_build_poly(hq, 4)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        pp.pp_build_poly(hq, 4, interval_ab=(0.1, 30.0))  # host work only
        o = pp.pp_default_opts()
        o.orth = pp.PP_ORTH_LANCZOS
        pp.pp_set_opts(hq, o)
        with pytest.raises(pp.PPError) as e:  # non-Hermitian complex: Arnoldi only
            pp.pp_apply(hq, pp.PP_SIGN, 1024, 2048)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(hq)
    h = pp.pp_create_stencil(pp.PP_LAPLACE3D7, (4, 4, 4))
    try:
        with pytest.raises(pp.PPError) as e:  # apply before build_poly
            pp.pp_apply(h, pp.PP_INVSQRT, 1, 2)
        assert e.value.status == pp.PP_ERR_STATE
        with pytest.raises(pp.PPError) as e:
            pp.pp_build_poly(h, -1)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:
            pp.pp_build_poly(h, 4, 9)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:
            pp.pp_build_poly(h, 4, interval_ab=(2.0, 1.0))
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:  # checked before the node run
            pp.pp_build_poly(h, 4, pp.PP_RITZ_LEJA, interval_ab=(0.0, 1.0))
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:
            pp.pp_get_poly_nodes(h)
        assert e.value.status == pp.PP_ERR_STATE
        pp.pp_build_poly(h, 4)
        # Chebyshev q: its nodes are the 5 first-kind Chebyshev nodes of [a,b],
        # in Leja order (the order of its Newton form)
        kind, x, _ = pp.pp_get_poly_nodes(h)
        _, (a, b), _ = pp.pp_get_poly(h)
        t = np.pi * (np.arange(5) + 0.5) / 5
        assert kind == pp.PP_CHEBYSHEV
        assert np.allclose(np.sort(x), np.sort(0.5 * (a + b) + 0.5 * (b - a) * np.cos(t)), rtol=1e-15)
        # reverse Leja order: the last node has the largest modulus, the one before the smallest
        assert x[-1] == x.max() and x[-2] == x.min()
        o = pp.pp_default_opts()
        o.clenshaw = 2
        with pytest.raises(pp.PPError) as e:
            pp.pp_set_opts(h, o)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:  # aliasing
            pp.pp_apply(h, pp.PP_INVSQRT, 1024, 1024)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:
            pp.pp_apply(h, 3, 1024, 2048)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        with pytest.raises(pp.PPError) as e:  # the sign function needs a Q^2 handle
            pp.pp_apply(h, pp.PP_SIGN, 1024, 2048)
        assert e.value.status == pp.PP_ERR_UNSUPPORTED
        with pytest.raises(pp.PPError) as e:
            pp.pp_apply(h, pp.PP_SQRT, 1024, 2048, m_max=0)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
        o = pp.pp_default_opts()
        o.precision = 7
        with pytest.raises(pp.PPError) as e:
            pp.pp_set_opts(h, o)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(h)
    # non-Hermitian CSR handles need an interval (Hermitian ones estimate it on the device)
    h = pp.pp_create_csr(16, 8, 8, 8, is_hermitian=False)
    try:
        with pytest.raises(pp.PPError) as e:
            pp.pp_build_poly(h, 4)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(h)

    pp.pp_destroy(None)


def test_autotune_degree_model():
    # F64 stencil handles: the degree choice needs no device work (closed-form
    # interval); the chosen degree is a candidate and q is built with it
    pp = load()
    cands = {0, 1, 2, 3, 4, 6, 8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128}
    for kind, dims in ((pp.PP_LAPLACE2D5, (1000, 1000)), (pp.PP_LAPLACE3D7, (100, 100, 100)),
                       (pp.PP_LAPLACE2D5, (12, 10))):
        h = pp.pp_create_stencil(kind, dims)
        try:
            d = pp.pp_autotune(h, 1e-9, 64)
            assert d in cands and d <= 64
            c, ab, img = pp.pp_get_poly(h)
            assert len(c) == d + 1
        finally:
            pp.pp_destroy(h)
    # harder problem (larger kappa) never gets a lower degree than an easy one of the same kind
    hs = [pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims) for dims in ((1000, 1000), (20, 20))]
    try:
        d_hard, d_easy = (pp.pp_autotune(h, 1e-9, 64) for h in hs)
        assert d_hard >= d_easy
        with pytest.raises(pp.PPError) as e:
            pp.pp_autotune(hs[0], 0.0, 64)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        for h in hs:
            pp.pp_destroy(h)


def reverse_units(x):
    """A node sequence reversed unit by unit: a conjugate pair (z, conj z) stays in that order."""
    x = list(np.atleast_1d(x))
    units, i = [], 0
    while i < len(x):
        if np.imag(x[i]) > 0:
            units.append(x[i:i + 2])
            i += 2
        else:
            units.append(x[i:i + 1])
            i += 1
    return np.array([z for u in units[::-1] for z in u])


def real_basis_eval(coef, x, z):
    """q(z) = sum_i coef_i R_i(z) in the real basis of pp_set_poly_nodes:
    R_0 = 1; a real node: R_{i+1} = (z - x_i) R_i; a pair (x_i, conj x_i):
    R_{i+1} = (z - Re x_i) R_i, R_{i+2} = (z - Re x_i) R_{i+1} + (Im x_i)^2 R_i."""
    z = np.asarray(z, dtype=complex)
    R_prev, R = np.zeros_like(z), np.ones_like(z)
    out = coef[0] * R
    i = 0
    while i + 1 < len(coef):
        if np.imag(x[i]) > 0:
            R1 = (z - x[i].real) * R
            out = out + coef[i + 1] * R1
            if i + 2 < len(coef):
                R2 = (z - x[i].real) * R1 + x[i].imag ** 2 * R
                out = out + coef[i + 2] * R2
                R_prev, R = R1, R2
            i += 2
        else:
            R_prev, R = R, (z - np.real(x[i])) * R
            out = out + coef[i + 1] * R
            i += 1
    return out


@pytest.mark.parametrize("nodes,ab", [
    ([0.7, 2.5, 1.1, 6.0, 3.3], (0.2, 7.0)),
    ([0.8, 1.5 + 0.7j, 1.5 - 0.7j, 3.0 + 1.2j, 3.0 - 1.2j, 5.0, 2.2], (0.2, 7.0)),
    ([2.0 + 1.0j, 2.0 - 1.0j], (1.0, 3.0)),
    ([4.0 - 0.5j, 1.0, 4.0 + 0.5j, 0.3 + 0.1j, 0.3 - 0.1j], (0.2, 7.0)),
], ids=["real5", "pairs7", "pair2", "pairs5"])
def test_set_poly_nodes_matches_oracle(nodes, ab):
    # host-only construction of q from given nodes: Leja order, Newton form in
    # the real basis, positivity, image; against the oracle's complex Newton form
    pp = load()
    z = np.array(nodes)
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (5, 4, 3), [0.5])
    try:
        pp.pp_set_poly_nodes(h, z, interval_ab=ab)
        kind, x, cap = pp.pp_get_poly_nodes(h)
        coef, abr, img = pp.pp_get_poly(h)
        assert kind == pp.PP_NODES and len(x) == len(z) and len(coef) == len(z)
        # the Newton form takes the nodes in reverse Leja order (pairs kept, Im > 0 first)
        xo = reverse_units(ritz.leja_order(z))
        assert np.allclose(x, xo, rtol=0, atol=0)
        ao = ritz.newton_coeffs(xo)
        pts = np.concatenate([np.linspace(ab[0], ab[1], 41), z, [1 + 2j, 3 - 1j]])
        assert np.allclose(real_basis_eval(coef, x, pts), ritz.newton_eval(ao, xo, pts), rtol=1e-12, atol=1e-14)
        assert np.allclose(real_basis_eval(coef, x, z), z ** -0.5, rtol=1e-12)
        # image of |z q(z)^2| on [a,b] and at the nodes
        t = np.concatenate([np.linspace(ab[0], ab[1], 20001), np.geomspace(ab[0], ab[1], 20001), z])
        qt = ritz.newton_eval(ao, xo, t)
        p = np.abs(t * qt * qt)
        assert img[0] == pytest.approx(p.min(), rel=1e-9) and img[1] == pytest.approx(p.max(), rel=1e-9)
        assert abr == ab
        assert cap == pytest.approx(0.25 * max(abs(a - b) for a in z for b in z), rel=1e-15)
    finally:
        pp.pp_destroy(h)


def test_set_poly_nodes_validation():
    pp = load()
    hl = pp.pp_create_stencil(pp.PP_LAPLACE2D5, (6, 5))
    hc = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (5, 4, 3), [0.5])
    try:
        bad = [(hl, [1.0, 2.0 + 1j, 2.0 - 1j], pp.PP_ERR_INVALID_ARG),   # complex nodes, Hermitian handle
               (hc, [1.0, 2.0 + 1j], pp.PP_ERR_INVALID_ARG),              # pair without conjugate
               (hc, [1.0, 2.0 + 1j, 2.0 - 0.5j], pp.PP_ERR_INVALID_ARG),
               (hc, [1.0, -0.5, 2.0], pp.PP_ERR_NONPRIMARY),              # Re <= 0
               (hc, [1.0, 2.0, 1.0], pp.PP_ERR_NONPRIMARY),               # coincident
               (hc, [], pp.PP_ERR_INVALID_ARG),
               (hc, list(np.linspace(1, 2, 130)), pp.PP_ERR_INVALID_ARG),
               (hc, [1.0, float("nan")], pp.PP_ERR_INVALID_ARG)]
        for h, z, st in bad:
            with pytest.raises(pp.PPError) as e:
                pp.pp_set_poly_nodes(h, np.array(z, dtype=complex if np.iscomplexobj(np.array(z)) else float))
            assert e.value.status == st, z
        # a linear interpolant of z^{-1/2} at 1 and 2 turns negative near 5.8:
        # positive on [0.5, 3], rejected on [0.5, 8]
        pp.pp_set_poly_nodes(hl, np.array([1.0, 2.0]), interval_ab=(0.5, 3.0))
        with pytest.raises(pp.PPError) as e:
            pp.pp_set_poly_nodes(hl, np.array([1.0, 2.0]), interval_ab=(0.5, 8.0))
        assert e.value.status == pp.PP_ERR_NONPRIMARY
        # default interval of a stencil handle: its closed form
        pp.pp_set_poly_nodes(hl, np.array([0.5, 3.0, 7.0]))
        _, ab, _ = pp.pp_get_poly(hl)
        assert ab == pytest.approx(ops.laplace_interval((6, 5)), rel=1e-14)
        with pytest.raises(pp.PPError) as e:
            pp.pp_build_poly(hl, 3, pp.PP_NODES)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(hl)
        pp.pp_destroy(hc)


@pytest.mark.parametrize("degree", [0, 3, 8, 16])
@pytest.mark.parametrize("ritz_values", [
    [1 + 0.5j, 1 - 0.5j, 3.0, 4 + 1j, 4 - 1j, 6.0, 0.2 + 0.3j, 0.2 - 0.3j],
    [2 + 3j, 2 - 3j, 10 + 0.1j, 10 - 0.1j, 5.0],
    [0.05, 2.0, 9.0],
], ids=["hull8", "hull5", "real3"])
def test_set_poly_lsq_matches_oracle(ritz_values, degree):
    # least-squares q on the oracle's contour points: the library's Newton
    # form (at Leja points of the contour) against the oracle's orthonormal
    # basis evaluation, on the contour and inside it
    pp = load()
    th = np.array(ritz_values, dtype=complex)
    z = lsq.contour(th, 0.5 * np.abs(th).min() if np.any(th.imag != 0) else 0.1, 400)
    P, H = lsq.basis(z, degree + 1)
    al = lsq.coeffs(P, z ** -0.5)
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (5, 4, 3), [0.5])
    try:
        pp.pp_set_poly_lsq(h, degree, z)
        kind, x, cap = pp.pp_get_poly_nodes(h)
        coef, ab, img = pp.pp_get_poly(h)
        assert kind == pp.PP_LSQ_CONTOUR and len(x) == degree + 1
        assert all(np.min(np.abs(z - xi)) == 0 for xi in np.atleast_1d(x))  # nodes are contour points
        inside = np.array([z.real.mean(), 0.5 * (z.real.min() + z.real.max()) + 0.1j * np.abs(z.imag).max()])
        pts = np.concatenate([z, inside])
        qo = lsq.evaluate(H, al, len(z), pts)
        ql = real_basis_eval(coef, np.atleast_1d(x), pts)
        assert np.abs(ql - qo).max() < 1e-9 * np.abs(qo).max()
        qz = qo[:len(z)]
        assert img[0] == pytest.approx(np.abs(z * qz * qz).min(), rel=1e-9)
        assert img[1] == pytest.approx(np.abs(z * qz * qz).max(), rel=1e-9)
    finally:
        pp.pp_destroy(h)


def test_lsq_validation_and_segment():
    pp = load()
    hl = pp.pp_create_stencil(pp.PP_LAPLACE2D5, (6, 5))
    hc = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, (5, 4, 3), [0.5])
    try:
        for h, z, st in [(hc, np.array([1.0 + 1j, 2.0, 3.0 - 0.5j]), pp.PP_ERR_UNSUPPORTED),  # not symmetric
                         (hl, np.array([1.0 + 1j, 1.0 - 1j, 3.0]), pp.PP_ERR_INVALID_ARG),    # complex, Hermitian
                         (hc, np.array([-1.0, 2.0, 3.0]), pp.PP_ERR_INVALID_ARG),             # on (-inf, 0]
                         (hc, np.array([1.0, 2.0]), pp.PP_ERR_INVALID_ARG)]:                  # N < degree + 1
            with pytest.raises(pp.PPError) as e:
                pp.pp_set_poly_lsq(h, 2, z)
            assert e.value.status == st
        # pp_build_poly with a known real spectrum: the least-squares q on its segment
        pp.pp_build_poly(hl, 6, pp.PP_LSQ_CONTOUR)
        coef, (a, b), _ = pp.pp_get_poly(hl)
        assert (a, b) == pytest.approx(ops.laplace_interval((6, 5)), rel=1e-14)
        kind, x, _ = pp.pp_get_poly_nodes(hl)
        seg = np.linspace(a, b, 2000)
        P, H = lsq.basis(seg, 7)
        al = lsq.coeffs(P, seg ** -0.5)
        t = np.linspace(a, b, 37)
        assert kind == pp.PP_LSQ_CONTOUR
        assert np.allclose(real_basis_eval(coef, x, t), lsq.evaluate(H, al, 2000, t), rtol=1e-9)
    finally:
        pp.pp_destroy(hl)
        pp.pp_destroy(hc)


def test_complex_nodes_newton_form_matches_oracle():
    # complex operator (Q^2 handle, host work only): unpaired complex nodes in
    # reverse Leja order, and the Newton coefficients of the interpolant of
    # z^{-1/2} at them (real parts b_i / cap^i = a_i) against the oracle
    pp = load()
    rng = np.random.default_rng(5)
    z = rng.uniform(0.5, 6.0, 9) + 1j * rng.uniform(-1.5, 1.5, 9)
    hq = pp.pp_create_stencil(pp.PP_WILSON4D_Q2, (4, 4, 4, 4), [-1.4, 0.3], links=64, dtype=pp.PP_C128)
    try:
        pp.pp_set_poly_nodes(hq, z)
        kind, x, cap = pp.pp_get_poly_nodes(hq)
        assert kind == pp.PP_NODES
        ref = ritz.leja_order(z, pairs=False)[::-1]
        assert np.array_equal(x, ref)
        a = ritz.newton_coeffs(ref)
        coef, _, _ = pp.pp_get_poly(hq)
        assert np.max(np.abs(coef - a.real)) < 1e-12 * np.max(np.abs(a))
        with pytest.raises(pp.PPError) as e:  # Re <= 0 is refused
            pp.pp_set_poly_nodes(hq, np.array([1.0 + 1j, -0.5 + 0.2j]))
        assert e.value.status == pp.PP_ERR_NONPRIMARY
    finally:
        pp.pp_destroy(hq)
