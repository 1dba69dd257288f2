"""GPU parity of the batched solver (pp_apply_batch, and pp_apply with
nrhs > 1) through the C ABI.

Every right-hand side of a batch is an independent Krylov process run in
lockstep with the others.  The batched kernels keep the single-vector
kernels' chunking and fixed-order reductions, so a process in a batch must
give the same iterate as pp_apply on that right-hand side alone; the tests
check that to 1e-14 and, separately, the results against the FP64 oracle at
1e-10 (the solve tolerance of the parity tests; mixed precision: within
max(3 x the double-word error, tol)).
"""
import numpy as np
import pytest

import synth
from oracle import exact, krylov, operators as ops
from tests.libpp import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"f64": 0, "dw": 1, "mixed": 2}


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


KIND = {"laplace2d5": 0, "laplace3d7": 1, "convdiff3d7": 2}


def make(pp, kind, dims, degree, prec, side=0, check_every=0):
    sk = {"laplace2d5": pp.PP_LAPLACE2D5, "laplace3d7": pp.PP_LAPLACE3D7,
          "convdiff3d7": pp.PP_CONVDIFF3D7_UPWIND}[kind]
    h = pp.pp_create_stencil(sk, dims, [0.5] if kind == "convdiff3d7" else None)
    pp.pp_build_poly(h, degree)
    o = pp.pp_default_opts()
    o.precision = PREC[prec]
    o.side = side
    o.check_every = check_every
    pp.pp_set_opts(h, o)
    return h


def exact_of(kind, dims, b, power):
    if kind == "laplace2d5" or kind == "laplace3d7":
        return exact.separable_fun(dims, b, power)
    A = ops.convdiff(dims, 0.5)
    if A.shape[0] <= 2000:
        return exact.dense_fun(A, b, power, hermitian=False)
    return krylov.plain_reference(A.dot, b, power, tol=1e-13, m_max=1500, k_chk=8)["x"]


@pytest.mark.parametrize("prec", ["f64", "dw"])
@pytest.mark.parametrize("kind,dims,degree", [("laplace3d7", (33, 17, 29), 8),
                                              ("convdiff3d7", (19, 23, 9), 4),
                                              ("laplace2d5", (64, 38), 9)])
def test_multi_rhs_equals_single(kind, dims, degree, prec):
    pp = load()
    h = make(pp, kind, dims, degree, prec)
    try:
        n = int(np.prod(dims))
        r = 3
        B = synth.rhs(n, 7, nrhs=r)  # (r, n): column-major n x r on the device
        bd = dev(B.reshape(-1))
        xd = torch.empty(r * n, dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, -1, bd, xd, m_max=300, tol=1e-12, nrhs=r)
        assert st.status == pp.PP_OK
        X = host(xd).reshape(r, n)
        for i in range(r):
            xs = torch.empty(n, dtype=torch.float64, device="cuda")
            pp.pp_apply(h, -1, dev(B[i]), xs, m_max=300, tol=1e-12)
            assert rel(X[i], host(xs)) < 1e-14
            assert rel(X[i], exact_of(kind, dims, B[i], -0.5)) < 1e-10
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["dw", "mixed"])
@pytest.mark.parametrize("side", [0, 1], ids=["left", "right"])
def test_heterogeneous_batch(side, prec):
    # four groups (degrees 4 / 8, Lanczos / CGS2), mixed f, uneven sizes and nrhs
    pp = load()
    spec = [("laplace2d5", (61, 37), 8, -1, 2), ("laplace3d7", (20, 21, 22), 4, 1, 1),
            ("convdiff3d7", (19, 23, 9), 8, 1, 3), ("convdiff3d7", (24, 20, 16), 4, -1, 2),
            ("laplace2d5", (40, 30), 8, 1, 1)]
    hs, bs, xs, Bs = [], [], [], []
    try:
        for i, (kind, dims, deg, f, r) in enumerate(spec):
            hs.append(make(pp, kind, dims, deg, prec, side))
            n = int(np.prod(dims))
            B = synth.rhs(n, 100 + i, nrhs=r) if r > 1 else synth.rhs(n, 100 + i)[None, :]
            Bs.append(B)
            bs.append(dev(B.reshape(-1)))
            xs.append(torch.empty(r * n, dtype=torch.float64, device="cuda"))
        stats = pp.pp_apply_batch(hs, [q[3] for q in spec], bs, xs, nrhs=[q[4] for q in spec],
                                  m_max=300, tol=1e-11)
        for i, (kind, dims, deg, f, r) in enumerate(spec):
            assert stats[i].status == pp.PP_OK
            X = host(xs[i]).reshape(r, -1)
            for q in range(r):
                ref = exact_of(kind, dims, Bs[i][q], 0.5 * f)
                err = rel(X[q], ref)
                if prec == "dw":
                    assert err < 1e-10, (i, q, err)
                else:
                    # the double-word solve of the same right-hand side
                    o = pp.pp_default_opts()
                    o.precision = PREC["dw"]
                    o.side = side
                    pp.pp_set_opts(hs[i], o)
                    y = torch.empty(X.shape[1], dtype=torch.float64, device="cuda")
                    pp.pp_apply(hs[i], f, dev(Bs[i][q]), y, m_max=300, tol=1e-11)
                    err_dw = rel(host(y), ref)
                    o.precision = PREC["mixed"]
                    pp.pp_set_opts(hs[i], o)
                    assert err <= max(3 * err_dw, 1e-11), (i, q, err, err_dw)
    finally:
        for h in hs:
            pp.pp_destroy(h)


def test_batch_zero_rhs_and_errors():
    pp = load()
    h1 = make(pp, "laplace2d5", (30, 20), 4, "dw")
    h2 = make(pp, "laplace3d7", (10, 12, 9), 4, "f64")
    try:
        n = 600
        B = synth.rhs(n, 3, nrhs=2)
        B[1] = 0.0
        bd = dev(B.reshape(-1))
        xd = torch.full((2 * n,), 5.0, dtype=torch.float64, device="cuda")
        st = pp.pp_apply_batch([h1], [-1], [bd], [xd], nrhs=[2], m_max=200, tol=1e-12)
        X = host(xd).reshape(2, n)
        assert st[0].status == pp.PP_OK and np.all(X[1] == 0.0)
        assert rel(X[0], exact.separable_fun((30, 20), B[0], -0.5)) < 1e-10
        # mismatched precision across the batch
        b2 = dev(synth.rhs(1080, 1))
        x2 = torch.empty(1080, dtype=torch.float64, device="cuda")
        with pytest.raises(pp.PPError) as e:
            pp.pp_apply_batch([h1, h2], [-1, -1], [dev(B[0]), b2], [xd[:n], x2], m_max=200, tol=1e-12)
        assert e.value.status == pp.PP_ERR_INVALID_ARG
    finally:
        pp.pp_destroy(h1)
        pp.pp_destroy(h2)


def test_batch_config_64_problems():
    # the 64-problem batch (n log-uniform in [1e3, 1e6], 1-16 right-hand sides,
    # mixed f): every process against pp_apply on its own right-hand side for a
    # sample of problems, and against the closed form for the Laplacians
    pp = load()
    probs = synth.batch_problems(64, seed=2)
    hs, bs, xs = [], [], []
    try:
        for i, p in enumerate(probs):
            hs.append(make(pp, p["kind"], p["dims"], 16, "dw"))
            n = int(np.prod(p["dims"]))
            B = synth.rhs(n, 1000 + i, nrhs=p["nrhs"]) if p["nrhs"] > 1 else synth.rhs(n, 1000 + i)[None, :]
            bs.append(dev(B.reshape(-1)))
            xs.append(torch.empty(p["nrhs"] * n, dtype=torch.float64, device="cuda"))
        stats = pp.pp_apply_batch(hs, [p["f"] for p in probs], bs, xs, nrhs=[p["nrhs"] for p in probs],
                                  m_max=400, tol=1e-10)
        assert all(s.status == pp.PP_OK for s in stats)
        rng = np.random.default_rng(0)
        for i in rng.choice(len(probs), 8, replace=False):
            p = probs[i]
            n = int(np.prod(p["dims"]))
            X = host(xs[i]).reshape(p["nrhs"], n)
            B = host(bs[i]).reshape(p["nrhs"], n)
            q = int(rng.integers(p["nrhs"]))
            y = torch.empty(n, dtype=torch.float64, device="cuda")
            pp.pp_apply(hs[i], p["f"], dev(B[q]), y, m_max=400, tol=1e-10)
            assert rel(X[q], host(y)) < 1e-14, (i, q)
            if p["kind"] != "convdiff3d7":
                assert rel(X[q], exact.separable_fun(p["dims"], B[q], 0.5 * p["f"])) < 1e-9, (i, q)
    finally:
        for h in hs:
            pp.pp_destroy(h)


def _oracle_batch_member(kind, dims, b, power):
    """x* for one process of the 64-problem batch: the closed form for the
    Laplacians and for convection-diffusion up to 20 points per direction
    (its diagonal similarity then has condition <= 1.5^{9.5} per direction),
    else the oracle's Algorithm 1 (Chebyshev degree 16, CGS2) to a stopping
    estimate of 1e-12 with its CSR products on all host cores."""
    if kind != "convdiff3d7":
        return exact.separable_fun(dims, b, power)
    if max(dims) <= 20:
        return exact.separable_fun(dims, b, power, "convdiff", 0.5)
    from oracle import chebyshev as cheb, spmv
    A = ops.convdiff(dims, 0.5)
    a, b_ = ops.convdiff_interval(dims, 0.5)
    r = krylov.pp_arnoldi(spmv.CsrMv(A), b, power, cheb.interp_coeffs(a, b_, 17), (a, b_), side="left",
                          m_max=300, tol=1e-12, k_chk=3, orth="cgs2")
    assert r["converged"]
    return r["x"]


def test_batch_config_64_problems_bench_arithmetic():
    # the configuration the batched bench times: mixed precision, the degree of
    # every problem chosen by pp_autotune, stopping estimate 1e-9, one
    # pp_apply_batch over the 64 problems; every process (problem, right-hand
    # side) against the FP64 oracle at the 1e-8 target of mixed precision
    pp = load()
    probs = synth.batch_problems(64, seed=2)
    hs, bs, xs, Bs, degs = [], [], [], [], []
    try:
        for i, p in enumerate(probs):
            sk = {"laplace2d5": pp.PP_LAPLACE2D5, "laplace3d7": pp.PP_LAPLACE3D7,
                  "convdiff3d7": pp.PP_CONVDIFF3D7_UPWIND}[p["kind"]]
            h = pp.pp_create_stencil(sk, p["dims"], [0.5] if p["kind"] == "convdiff3d7" else None)
            hs.append(h)
            o = pp.pp_default_opts()
            o.precision = PREC["mixed"]
            pp.pp_set_opts(h, o)
            degs.append(pp.pp_autotune(h, 1e-9, 64))
            n = int(np.prod(p["dims"]))
            B = synth.rhs(n, 1000 + i, nrhs=p["nrhs"]) if p["nrhs"] > 1 else synth.rhs(n, 1000 + i)[None, :]
            Bs.append(B)
            bs.append(dev(B.reshape(-1)))
            xs.append(torch.empty(p["nrhs"] * n, dtype=torch.float64, device="cuda"))
        assert len(set(degs)) >= 1
        stats = pp.pp_apply_batch(hs, [p["f"] for p in probs], bs, xs, nrhs=[p["nrhs"] for p in probs],
                                  m_max=1000, tol=1e-9)
        assert all(s.status == pp.PP_OK for s in stats)
        # the oracle's x* of every process; the large convection-diffusion ones in spawned workers
        from tests.oracle_pool import convdiff_solve, map_spawn
        jobs, slots, refs = [], [], {}
        for i, p in enumerate(probs):
            for q in range(p["nrhs"]):
                if p["kind"] == "convdiff3d7" and max(p["dims"]) > 20:
                    jobs.append((tuple(p["dims"]), Bs[i][q], 0.5 * p["f"]))
                    slots.append((i, q))
                else:
                    refs[(i, q)] = _oracle_batch_member(p["kind"], p["dims"], Bs[i][q], 0.5 * p["f"])
        for key, x in zip(slots, map_spawn(convdiff_solve, jobs)):
            refs[key] = x
        for i, p in enumerate(probs):
            X = host(xs[i]).reshape(p["nrhs"], -1)
            for q in range(p["nrhs"]):
                err = rel(X[q], refs[(i, q)])
                assert err < 1e-8, (i, q, p["kind"], p["dims"], degs[i], err)
    finally:
        for h in hs:
            pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["f64", "dw", "mixed"])
def test_csr_block_spmm_right_hand_sides(prec):
    # nrhs > 1 on CSR handles runs the right-hand sides of each matrix as one
    # lockstep group (block SpMM operator steps, up to 16 per group): every
    # column against its single-vector solve (bitwise in FP64 and
    # double-word, the same kernels and the handle's own quadrature) and
    # against the FP64 oracle
    pp = load()
    cases = [("laplace2d5", (30, 23), -1, 6, 20, True),     # Hermitian, Lanczos, 16 + 4 columns
             ("convdiff3d7", (11, 9, 8), 1, 5, 5, False)]   # non-Hermitian, CGS2
    for kind, dims, f, degree, r, herm in cases:
        rp, col, val = synth.stencil_csr(kind, dims, 0.5 if kind == "convdiff3d7" else 0.0)
        keep = [dev(a) for a in (rp, col, val)]
        n = int(np.prod(dims))
        h = pp.pp_create_csr(n, *keep, is_hermitian=herm)
        try:
            ab = ops.laplace_interval(dims) if kind != "convdiff3d7" else ops.convdiff_interval(dims, 0.5)
            pp.pp_build_poly(h, degree, interval_ab=ab)
            o = pp.pp_default_opts()
            o.precision = PREC[prec]
            pp.pp_set_opts(h, o)
            B = np.stack([synth.rhs(n, 40 + s) for s in range(r)], axis=0)
            X = torch.empty((r, n), dtype=torch.float64, device="cuda")
            st = pp.pp_apply(h, f, dev(B), X, m_max=300, tol=1e-11, nrhs=r)
            assert st.status == pp.PP_OK
            Xh = host(X)
            for k in range(r):
                ref = exact.separable_fun(dims, B[k], 0.5 * f, "laplace" if kind != "convdiff3d7" else "convdiff",
                                          0.5 if kind == "convdiff3d7" else 0.0)
                assert rel(Xh[k], ref) < (1e-10 if prec != "mixed" else 1e-8), (kind, k)
                if prec != "mixed":
                    xk = torch.empty(n, dtype=torch.float64, device="cuda")
                    pp.pp_apply(h, f, dev(B[k].copy()), xk, m_max=300, tol=1e-11)
                    assert np.array_equal(Xh[k], host(xk)), (kind, k)
        finally:
            pp.pp_destroy(h)


def test_csr_block_spmm_graph_laplacian():
    # Example 3's problem class with several right-hand sides: L^{1/2} e_i for
    # three canonical vectors of the synthetic directed graph in one call
    pp = load()
    from tests.test_gpu_graph import N, graph, reference
    rp, col, val = graph()
    keep = [dev(a) for a in (rp, col, val)]
    h = pp.pp_create_csr(N, *keep, is_hermitian=False)
    try:
        pp.pp_build_poly(h, 7, pp.PP_HARMONIC_RITZ)
        o = pp.pp_default_opts()
        o.precision = PREC["dw"]
        pp.pp_set_opts(h, o)
        seeds = (4, 9, 11)
        B = np.stack([reference(s)[0] for s in seeds], axis=0)
        X = torch.empty((3, N), dtype=torch.float64, device="cuda")
        st = pp.pp_apply(h, pp.PP_SQRT, dev(B), X, m_max=800, tol=1e-11, nrhs=3)
        assert st.status == pp.PP_OK
        Xh = host(X)
        for k, s in enumerate(seeds):
            assert rel(Xh[k], reference(s)[1]) < 1e-7
    finally:
        pp.pp_destroy(h)


@pytest.mark.parametrize("prec", ["dw", "mixed"])
def test_batch_plan_graph_replays(prec):
    # a batch plan solves repeatedly with its segment graphs: the first solve
    # captures them, later ones replay them; every solve equals the one-shot
    # pp_apply_batch (direct launches) bit for bit, for new right-hand sides too
    pp = load()
    spec = [("laplace2d5", (41, 37), 6, -1, 3), ("convdiff3d7", (13, 11, 9), 6, 1, 2),
            ("laplace3d7", (12, 10, 9), 3, 1, 1)]
    hs = [make(pp, k, d, deg, prec) for k, d, deg, f, r in spec]
    try:
        fs = [q[3] for q in spec]
        nr = [q[4] for q in spec]
        plan = pp.pp_batch_create(hs, fs, nrhs=nr, m_max=300)
        try:
            for seed in (7, 8, 7):
                Bs = [synth.rhs(int(np.prod(d)), seed + i, nrhs=r).reshape(-1) if r > 1
                      else synth.rhs(int(np.prod(d)), seed + i) for i, (k, d, deg, f, r) in enumerate(spec)]
                bs = [dev(B) for B in Bs]
                xp = [torch.empty_like(b) for b in bs]
                xo = [torch.empty_like(b) for b in bs]
                st = pp.pp_batch_apply(plan, bs, xp, tol=1e-11)
                so = pp.pp_apply_batch(hs, fs, bs, xo, nrhs=nr, m_max=300, tol=1e-11)
                assert all(q.status == pp.PP_OK for q in st + so)
                for a, b in zip(xp, xo):
                    assert np.array_equal(host(a), host(b))
                assert [q.iters for q in st] == [q.iters for q in so]
            # a changed q invalidates the plan
            pp.pp_build_poly(hs[0], 5)
            with pytest.raises(pp.PPError) as e:
                pp.pp_batch_apply(plan, bs, xp, tol=1e-11)
            assert e.value.status == pp.PP_ERR_STATE
        finally:
            pp.pp_batch_destroy(plan)
    finally:
        for h in hs:
            pp.pp_destroy(h)
