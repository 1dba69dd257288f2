#!/usr/bin/env python3
"""Throughput of polynomially preconditioned f(A)b on GB300.

One step = one complete solve.  Default workload: x = A^{1/2} b
(Algorithm 1 with A^{1/2} b = A^{-1/2}(A b)) of the 3D upwind
convection-diffusion operator on a 128^3 grid (n = 2,097,152, c*h = 0.5,
non-Hermitian, so Arnoldi with CGS2), Chebyshev q of degree 16 on the exact
spectral interval, stopping estimate < 1e-10, mixed precision (double-word
start, FP32 once its rounding is below the tolerance).  --workload selects
the other single-GPU workloads.  The metric is solves per second over all
ranks; ranks solve independent right-hand sides (seed 0 + rank), no
collective on the data path.

Besides the timed value the line carries, measured outside the timed region:
accuracy.rel_err_vs_oracle (the timed solve's x against the FP64 oracle's
x*), the same configuration in the other arithmetics (companions: double-word
and IEEE FP64, each with its own oracle error), the degree-0 in-GPU baselines
(plain_gpu), the chain's roofline (live, and out of L2 on an 8192^2 grid),
the oracle's own whole solve on the host cores (cpu_baseline) and an
end-to-end figure through pp_apply_host.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload instead.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "f(A)b solves/sec and SpMV-chain HBM GB/s (% roofline) at 1e-8 rel err vs FP64 oracle"

# name -> (description, operator, grid, func (+1 sqrt / -1 invsqrt), degree, tol, orth)
WORKLOADS = {
    "convdiff128": ("3D convection-diffusion 128^3 upwind 7-point (n=2097152, c*h=0.5), f=A^(1/2), "
                    "Arnoldi with classical Gram-Schmidt twice, second pass delayed one step (DCGS2)",
                    "convdiff3d7", (128, 128, 128), 1, 16, 1e-10, "dcgs2"),
    "convdiff256": ("3D convection-diffusion 256^3 upwind 7-point (n=16777216, c*h=0.5; vectors of 67 MB in FP32: "
                    "the chain out of L2), f=A^(1/2), Arnoldi DCGS2, the default workload at 8x the size; basis capped at "
                    "100 columns (42 iterations)",
                    "convdiff3d7", (256, 256, 256), 1, 16, 1e-10, "dcgs2"),
    "laplace2048": ("2D Laplacian 2048^2 5-point matrix-free (n=4194304), f=A^(-1/2), Lanczos; "
                    "1e-8 target, estimate tolerance 1e-9", "laplace2d5", (2048, 2048), -1, 16, 1e-9,
                    "lanczos"),
    "laplace8192": ("2D Laplacian 8192^2 5-point matrix-free (n=67108864, vectors of 268 MB in FP32: out of "
                    "L2), f=A^(-1/2), Lanczos, degree 16, two-pass (basis memory O(n)); the out-of-L2 roofline "
                    "case of the 2048^2 configuration (use --probe for the per-step chain numbers)",
                    "laplace2d5", (8192, 8192), -1, 16, 1e-9, "lanczos"),
    "laplace64csr": ("2D Laplacian 64^2 5-point CSR (n=4096), f=A^(-1/2), Lanczos, degree 8",
                     "laplace2d5csr", (64, 64), -1, 8, 1e-10, "lanczos"),
    "batch64": ("64 independent problems in one batched call: 2D/3D Laplacians and 3D convection-diffusion, "
                "n log-uniform in [1e3, 1e6], 1-16 right-hand sides each, mixed sqrt / inverse sqrt (problem "
                "list seed 2); degree and stencil tile chosen by the autotuner; a solve = one right-hand side",
                "batch", (), 0, 0, 1e-9, "mixed"),
    "graph282k": ("L^(1/2) b, L = D_in - A the in-degree Laplacian of a synthetic directed power-law graph "
                  "(n=281903, 2312497 edges, in/out-degree exponents 2.1/2.7, graph seed 3; the size of "
                  "Example 3's web graph), non-Hermitian CSR, b = e_i (seed 4), Ritz polynomial of degree 15 "
                  "(d = 16), Arnoldi CGS2, stopping check every 32/d = 2 iterations; 1e-7 target, estimate "
                  "tolerance 1e-8", "graphcsr", (281903,), 1, 15, 1e-8, "cgs2"),
    "wilson16x32": ("A = D^H D, Wilson-type D on a periodic 16^3x32 lattice (n=1572864 complex), Haar "
                    "SU(3) links seed 1, m0=0.1, f=A^(-1/2), Lanczos; 1e-8 target, estimate tolerance 1e-9",
                    "wilson4d", (16, 16, 16, 32), -1, 16, 1e-9, "lanczos"),
    "sign16x32": ("sign(Q) b = Q (Q^2)^(-1/2) b, Q = Gamma_5 D_w(m_w=-1.4, mu=0.3) non-Hermitian (chemical "
                  "potential on the 32-site direction), periodic 16^3x32 lattice (n=1572864 complex), Haar SU(3) "
                  "links seed 1; complex Arnoldi CGS2, Ritz polynomial of degree 31 (d = 32), stopping check "
                  "every 64/d = 2 iterations; 1e-8 estimate tolerance", "wilsonq2", (16, 16, 16, 32), 2, 31,
                  1e-8, "cgs2"),
    "sign32x64": ("sign(Q) b as sign16x32 on the 32^3x64 lattice of Sec. 6, Example 2 (n=25165824 complex), "
                  "Ritz polynomial of degree 63 (d = 64), stopping check every iteration; 1e-8 estimate "
                  "tolerance", "wilsonq2", (32, 32, 32, 64), 2, 63, 1e-8, "cgs2"),
}
WILSON_M0 = 0.1
SIGN_MW, SIGN_MU = -1.4, 0.3  # Sec. 6, Example 2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="convdiff128", choices=sorted(WORKLOADS))
    p.add_argument("--degree", type=int, default=None, help="default: the workload's")
    p.add_argument("--prec", default="mixed", choices=["dw", "f64", "mixed"])
    p.add_argument("--tol", type=float, default=None, help="default: the workload's")
    p.add_argument("--m-max", type=int, default=None,
                   help="basis size cap (default 1000; 200 for sign32x64, whose vectors are 403 MB; 100 for convdiff256)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the degree-0 in-GPU baselines")
    p.add_argument("--no-companions", action="store_true",
                   help="skip the double-word / FP64 solves of the same configuration")
    p.add_argument("--no-oracle-err", action="store_true", help="skip the error against the FP64 oracle")
    p.add_argument("--no-out-of-l2", action="store_true", help="skip the 8192^2 out-of-L2 chain timing")
    p.add_argument("--plain-m-max", type=int, default=1000)
    p.add_argument("--poly", default=None, choices=["ritz", "harmonic", "lsq"],
                   help="graph workload: the kind of q (default ritz)")
    p.add_argument("--probe", action="store_true",
                   help="per-launch timing of the operator kernels on the workload (no bench line)")
    p.add_argument("--clenshaw", action="store_true",
                   help="evaluate q by the Chebyshev Clenshaw recurrence instead of the Newton/Horner form")
    p.add_argument("--two-pass", action="store_true",
                   help="two-pass Lanczos (O(n) basis memory, twice the operator passes)")
    p.add_argument("--autotune", action="store_true", help="degree and tile from pp_autotune")
    p.add_argument("--halo", action="store_true",
                   help="FP32 stencil Horner steps two per launch through TMA-staged halo tiles (opts.halo)")
    p.add_argument("--orth", default=None, choices=["cgs2", "dcgs2"],
                   help="Gram-Schmidt of the Arnoldi workloads (default: the workload's)")
    a = p.parse_args()
    w = WORKLOADS[a.workload]
    a.desc, a.kind, a.dims, a.func = w[0], w[1], w[2], w[3]
    a.degree = w[4] if a.degree is None else a.degree
    a.tol = w[5] if a.tol is None else a.tol
    if a.m_max is None:  # the 256^3 and 32^3 x 64 bases would not need 1000 columns (tens of GB each)
        a.m_max = {"sign32x64": 200, "convdiff256": 100}.get(a.workload, 1000)
    if a.orth is not None and w[6] not in ("cgs2", "dcgs2"):
        p.error("--orth applies to the Arnoldi workloads only")
    a.orth = w[6] if a.orth is None else a.orth
    a.n = 1
    for d in a.dims:
        a.n *= d
    if a.kind == "batch":
        a.n = 0
    a.complex = a.kind in ("wilson4d", "wilsonq2")
    if a.complex:
        a.n *= 12  # complex components per site
    return a


def max_over_ranks(x, ws):
    """The largest x over the ranks (an all-reduce MAX on the process group's
    device: CUDA under NCCL, host under gloo); x itself for one rank."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(steps, ws, t_max):
    """Whole-job solves/s of ws replicas that each ran `steps` solves, timed by
    the slowest rank (weak scaling, no collective on the data path)."""
    return ws * steps / t_max


_GRAPH = {}


def graph_csr(n):
    """CSR arrays of the synthetic web-graph Laplacian (built once per process)."""
    if n not in _GRAPH:
        import synth
        src, dst = synth.directed_powerlaw_graph(n, 2312497 if n == 281903 else 8 * n, seed=3)
        _GRAPH[n] = synth.graph_laplacian_csr(n, src, dst)
    return _GRAPH[n]


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def config(args, ws):
    return {"workload": args.desc + (" (degree and tile autotuned)" if args.autotune else "")
            + (", two-pass Lanczos" if args.two_pass else ""),
            "grid": list(args.dims), "n": args.n,
            "ch": 0.5 if args.kind == "convdiff3d7" else 0.0,
            "func": {1: "sqrt", -1: "invsqrt", 2: "sign"}[args.func],
            "poly": ({"ritz": "ritz (leja/newton)", "harmonic": "harmonic ritz (leja/newton)",
                      "lsq": "least squares on the Ritz-value contour"}[args.poly or "ritz"]
                     if args.kind in ("graphcsr", "wilsonq2") else "chebyshev"), "degree": args.degree,
            "q_eval": "clenshaw" if args.clenshaw else "newton-horner at Leja-ordered nodes",
            "side": "left", "orth": args.orth, "tol": args.tol, "rhs_per_rank": 1,
            "fp32_stencil_steps": "two per launch, TMA-staged halo tiles" if args.halo else "one per launch",
            "parallelism": f"replicas{ws}", "l2": "flushed between timed steps (256 MB write)"}


# ---------------------------------------------------------------- oracle (CPU)

class _OutOfBudget(Exception):
    pass


def oracle_problem(args, seed=0):
    """The oracle's operator (x -> A x on all host cores through the oracle's
    OpenMP CSR product) and right-hand side for the workload."""
    from oracle import operators as ops, spmv
    import synth
    P = {}
    if args.kind == "convdiff3d7":
        A = ops.convdiff(args.dims, 0.5)
        P["ab"] = ops.convdiff_interval(args.dims, 0.5)
        P["mv"], P["rhs"] = spmv.CsrMv(A), synth.rhs(A.shape[0], seed)
    elif args.kind == "wilson4d":
        from oracle import wilson
        D = wilson.dirac_matrix(args.dims, synth.wilson_links(args.dims, 1), WILSON_M0)
        mD, mDH = spmv.CsrMv(D), spmv.CsrMv(D.conj().T.tocsr())
        P["mv"] = lambda v: mDH(mD(v))  # noqa: E731
        P["ab"] = (0.01, 96.0)  # shapes q only; the cost per iteration does not depend on it
        P["rhs"] = synth.spinor_field(args.dims, seed)
    elif args.kind == "wilsonq2":
        from oracle import wilson
        mQ = spmv.CsrMv(wilson.q_matrix(args.dims, synth.wilson_links(args.dims, 1), SIGN_MW, SIGN_MU))
        P["Q"] = mQ
        P["mv"] = lambda v: mQ(mQ(v))  # noqa: E731
        P["rhs"] = synth.spinor_field(args.dims, seed)
    elif args.kind == "graphcsr":
        import scipy.sparse as sp
        rp, col, val = graph_csr(args.dims[0])
        A = sp.csr_matrix((val, col, rp), shape=(args.dims[0], args.dims[0]))
        P["mv"], P["rhs"] = spmv.CsrMv(A), synth.unit_vector(A.shape[0], 4 + seed)
    else:
        A = ops.laplace(args.dims)
        P["ab"] = ops.laplace_interval(args.dims)
        P["mv"], P["rhs"] = spmv.CsrMv(A), synth.rhs(A.shape[0], seed)
    return P


def oracle_timed(args, m_max, tol, seed=0, budget_s=None, P=None, max_iters=None):
    """Run the FP64 oracle (Algorithm 1, as it stands) on the workload and time it.

    Returns (result or None, set-up seconds, per-iteration seconds).  With
    budget_s the run is abandoned (result None) once it has taken longer."""
    from oracle import chebyshev as cheb, krylov
    if P is None:
        P = oracle_problem(args, seed)
    mv, rhs = P["mv"], P["rhs"]
    # delayed reorthogonalization builds the CGS2 basis in exact arithmetic: the oracle runs CGS2
    orth = "cgs2" if args.orth == "dcgs2" else args.orth
    stamps = []
    t0 = time.perf_counter()

    def hook(j):
        stamps.append(time.perf_counter())
        if budget_s is not None and stamps[-1] - t0 > budget_s:
            raise _OutOfBudget()
        if max_iters is not None and len(stamps) > max_iters:
            raise _OutOfBudget()

    r = None
    try:
        if args.kind == "graphcsr":  # Example 3: q from the oracle's own Ritz values (part of the set-up)
            from oracle import ritz
            n = rhs.shape[0]
            if args.poly == "lsq":
                from oracle import lsq
                H60, _ = ritz.arnoldi(mv, ritz.start_vector(n), max(60, args.degree + 1))
                th = ritz.ritz_values(H60, hermitian=False)
                th = th[np.abs(th) > 1e-4 * np.abs(th).max()]  # the null space of the singular L left out
                z = lsq.contour(th, 0.5 * np.abs(th).min(), max(2000, 20 * (args.degree + 1)))
                Pz, Hq = lsq.basis(z, args.degree + 1)
                al = lsq.coeffs(Pz, z ** -0.5)
                qf = (args.degree, lambda v: lsq.apply(mv, Hq, al, len(z), v))
            else:
                x, an = ritz.ritz_poly(mv, n, args.degree, harmonic=args.poly == "harmonic", hermitian=False)
                qf = (args.degree, lambda v: ritz.newton_apply(mv, an, x, v))
            r = krylov.pp_arnoldi(mv, rhs, 0.5 * args.func, q=qf, side="left", m_max=m_max, tol=tol,
                                  k_chk=max(1, 32 // (args.degree + 1)), orth=orth, on_iter=hook)
        elif args.kind == "wilsonq2":  # Example 2: complex Ritz q (set-up), (Q^2)^{-1/2} b, then Q
            from oracle import ritz, sign
            x, an = ritz.ritz_poly(mv, rhs.shape[0], args.degree, complex_=True, hermitian=False)
            qf = (args.degree, lambda v: ritz.newton_apply(mv, an, x, v))
            xs, r = sign.sign_krylov(P["Q"], rhs, q=qf, side="left", m_max=m_max, tol=tol,
                                     k_chk=max(1, 64 // (args.degree + 1)), orth=orth, on_iter=hook)
            r = dict(r, x=xs)
        else:
            a, b = P["ab"]
            c = cheb.interp_coeffs(a, b, args.degree + 1)
            r = krylov.pp_arnoldi(mv, rhs, 0.5 * args.func, c, (a, b), side="left", m_max=m_max, tol=tol,
                                  k_chk=max(1, 64 // (args.degree + 1)), hermitian=orth == "lanczos",
                                  orth=orth, on_iter=hook)
    except _OutOfBudget:
        r = None
    t_end = time.perf_counter()
    setup = stamps[0] - t0 if stamps else t_end - t0
    iters = [b_ - a_ for a_, b_ in zip(stamps[:-1], stamps[1:])]
    if r is not None:
        r["solve_s"] = t_end - t0
    return r, setup, iters


def oracle_threads():
    from oracle import spmv
    return spmv.threads()


# iterations of the GPU solve of the workloads whose oracle solve takes minutes
# (measured), to extrapolate the oracle's solve time from its iteration time
GPU_ITERS = {"laplace2048": 300, "wilson16x32": 6, "sign16x32": 8}

ORACLE_SAMPLE_NOTE = ("numpy/scipy FP64; CSR products on {t} OpenMP threads (the oracle's own kernel), "
                      "Gram-Schmidt products in OpenBLAS, vector updates in numpy")


def cpu_sample(args, m_full, budget_s=45.0):
    """The oracle on the full workload: whole solves at the bench's tolerance
    when one fits in budget_s, else the iterations run by then, extrapolated
    to m_full iterations.  Returns (cpu_baseline dict, the last whole run or None)."""
    t = oracle_threads()
    note = ORACLE_SAMPLE_NOTE.format(t=t)
    P = oracle_problem(args, 0)
    r, setup, iters = oracle_timed(args, 1000 if args.kind != "wilsonq2" else args.m_max, args.tol,
                                   budget_s=budget_s, P=P)
    if r is not None:
        return ({"value": 1.0 / r["solve_s"], "unit": "solves/s", "cores": t, "kind": "oracle",
                 "sample": f"one whole oracle solve of the full workload (Algorithm 1, {note}) to the "
                           f"bench's tolerance: set-up {setup:.2f}s + {r['iters']} iterations = "
                           f"{r['solve_s']:.1f}s"}, r)
    t_iter = statistics.mean(iters) if iters else float("nan")
    t_solve = setup + m_full * t_iter
    return ({"value": 1.0 / t_solve, "unit": "solves/s", "cores": t, "kind": "oracle",
             "sample": f"oracle Algorithm 1 ({note}) on the full workload, stopped after {budget_s:.0f}s: "
                       f"set-up {setup:.2f}s + {len(iters)} iterations of {t_iter:.2f}s, extrapolated to the "
                       f"{m_full} iterations of the GPU solve = {t_solve:.1f}s"}, None)


def oracle_reference(args, seed=0, run=None):
    """The FP64 oracle's x* for the workload's right-hand side (seed), or None.

    Laplacians: the closed form (sine basis).  Convection-diffusion and the
    graph Laplacian: the oracle's Algorithm 1 run to a tight stopping estimate
    (run, the cpu_baseline's whole solve, is reused when its estimate already
    met that).  Returns (x or None, description)."""
    import synth
    from oracle import exact
    if args.kind in ("laplace2d5", "laplace2d5csr"):
        if args.n > 5_000_000:
            return None, "not computed: the closed form needs dense 1D transforms of the 8192-point axes"
        b = synth.rhs(args.n, seed)
        return exact.separable_fun(args.dims, b, 0.5 * args.func, "laplace"), \
            "closed form (Kronecker product of 1D sine transforms)"
    tight = {"convdiff3d7": 1e-13, "graphcsr": 1e-11}.get(args.kind)
    if tight is None:
        return None, ("not computed by the bench (the oracle takes minutes per solve on the lattice); "
                      "the GPU tests compare this size with the free-field closed form")
    if run is not None and run.get("history") and run["history"][-1][1] < tight and seed == 0:
        r = run
    else:
        r, _, _ = oracle_timed(args, 1000, tight, seed)
    return r["x"], (f"oracle Algorithm 1 (FP64, {'Ritz' if args.kind == 'graphcsr' else 'Chebyshev'} q of "
                    f"degree {args.degree}, {'cgs2' if args.orth == 'dcgs2' else args.orth}) to a stopping estimate of "
                    f"{r['history'][-1][1]:.1e} < {tight:g} ({r['iters']} iterations)")


def accuracy_target(args):
    """The relative error the workload's result must meet: Example 3's 1e-7 for
    the graph Laplacian, the metric's 1e-8 for mixed precision and for the
    workloads quoted at 1e-8, 1e-10 for the FP64-grade runs of the others."""
    if args.kind == "graphcsr":
        return 1e-7
    if args.prec == "mixed" or args.workload in ("laplace2048", "laplace8192", "wilson16x32", "sign16x32",
                                                  "sign32x64"):
        return 1e-8
    return 1e-10


def rel_err(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def cpu_sample_batch(args, probs, budget_s=15.0):
    """The oracle (Algorithm 1, FP64) on one right-hand side of each problem of
    the batch's list, in list order, until about budget_s seconds of work."""
    from oracle import chebyshev as cheb, krylov, operators as ops, spmv
    import synth
    solved, t_used, used = 0, 0.0, []
    for i, p in enumerate(probs):
        dims = p["dims"]
        if p["kind"] == "convdiff3d7":
            A, ab = ops.convdiff(dims, 0.5), ops.convdiff_interval(dims, 0.5)
        else:
            A, ab = ops.laplace(dims), ops.laplace_interval(dims)
        deg = 16
        c = cheb.interp_coeffs(ab[0], ab[1], deg + 1)
        b = synth.rhs(A.shape[0], 1000 + i, nrhs=p["nrhs"]) if p["nrhs"] > 1 else synth.rhs(A.shape[0], 1000 + i)[None, :]
        mv = spmv.CsrMv(A)
        t0 = time.perf_counter()
        krylov.pp_arnoldi(mv, b[0], 0.5 * p["f"], c, ab, side="left", m_max=1000, tol=args.tol,
                          k_chk=max(1, 64 // (deg + 1)), hermitian=p["kind"] != "convdiff3d7",
                          orth="lanczos" if p["kind"] != "convdiff3d7" else "cgs2")
        t_used += time.perf_counter() - t0
        solved += 1
        used.append(i)
        if t_used > budget_s:
            break
    t = oracle_threads()
    return {"value": solved / t_used, "unit": "solves/s", "cores": t, "kind": "oracle", "solves": solved,
            "sample": f"oracle Algorithm 1 ({ORACLE_SAMPLE_NOTE.format(t=t)}, degree 16) on one right-hand side "
                      f"of each of problems {used[0]}..{used[-1]} of the batch's list ({solved} solves, "
                      f"{t_used:.1f}s)"}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.

    A step is one whole oracle solve where one takes at most a minute, else
    one oracle iteration (step_unit says which); warm-up: one step."""
    rank, ws, _ = dist_env()
    if rank != 0:
        return
    why = {"laplace8192": "the oracle's Krylov basis for 67M unknowns (537 MB per vector) does not fit host "
                          "memory; laplace8192 is the out-of-L2 probe of laplace2048, whose reference arm runs",
           "sign32x64": "one oracle iteration on 25M complex unknowns is 127 sparse Q^2 products of many minutes "
                        "each; sign16x32 (the same operator on the 16^3x32 lattice) has the reference arm"}
    if args.workload in why:
        print(json.dumps({"impl": "reference", "unavailable": why[args.workload]}), flush=True)
        return
    t = oracle_threads()
    note = ORACLE_SAMPLE_NOTE.format(t=t)
    budget = 150.0  # seconds of timed oracle work
    if args.kind == "batch":  # the oracle on one right-hand side of each problem, in list order
        import synth
        probs = synth.batch_problems(64, seed=2)
        cpu_sample_batch(args, probs, budget_s=5.0)  # warm-up
        cb = cpu_sample_batch(args, probs, budget_s=15.0)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "solves/s", "n_gpus": ws,
                "steps": cb["solves"], "warmup": 1, "ms_per_step": 1e3 / cb["value"],
                "step_unit": "one oracle solve of one right-hand side of a problem of the list",
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (problem list seed 2, b ~ N(0,1) seed 1000 + i)",
                "config": {"workload": args.desc, "problems": len(probs),
                           "right_hand_sides": sum(p["nrhs"] for p in probs),
                           "rows_total": sum(int(np.prod(p["dims"])) * p["nrhs"] for p in probs),
                           "tol": args.tol, "parallelism": "replicas1",
                           "l2": "flushed between timed steps (256 MB write)"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    P = oracle_problem(args, 0)
    t_run0 = time.perf_counter()
    # warm-up: one whole solve if it ends within a minute
    r, setup, its = oracle_timed(args, 1000, args.tol, budget_s=60.0, P=P)
    if r is not None:  # steps are whole solves, until the budget or --steps is reached
        times, m = [], r["iters"]
        while len(times) < max(1, args.steps) and (not times or sum(times) + statistics.mean(times) <= budget):
            r, _, _ = oracle_timed(args, 1000, args.tol, P=P)
            times.append(r["solve_s"])
        step_s, steps = statistics.mean(times), len(times)
        value = 1.0 / step_s
        unit = f"one whole oracle solve (set-up + {m} iterations)"
        sample = f"{steps} whole oracle solves of the full workload (Algorithm 1, {note}), one warm-up solve before"
    else:  # steps are oracle iterations: one run, stopped once warm-up + steps iterations are seen
        r, setup, its = oracle_timed(args, 1000, args.tol, budget_s=budget, P=P,
                                     max_iters=1 + max(1, args.steps))
        times = its[1:] or its
        step_s, steps = statistics.mean(times), len(times)
        m = GPU_ITERS.get(args.workload, r["iters"] if r is not None else None)
        value = 1.0 / (setup + m * step_s)
        unit = "one oracle iteration"
        sample = (f"{steps} oracle iterations (after one warm-up iteration) on the full workload (Algorithm 1, "
                  f"{note}); value = 1 / (set-up {setup:.1f}s + {m} iterations of {step_s:.2f}s), {m} being "
                  f"the GPU solve's iteration count")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": steps, "warmup": 1, "ms_per_step": 1e3 * step_s, "step_unit": unit,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (b ~ N(0,1), seed 0)", "config": config(args, 1),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": t, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_iters": m, "run_s": time.perf_counter() - t_run0}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


ST_STEP_END = b"// The flat block index is mapped"  # ops.cu: the batched kernel starts here


def st_step_source_hash(kernel_src):
    """Hash of ops.cu up to the batched kernel: the stencil helpers and st_step."""
    data = open(kernel_src, "rb").read()
    cut = data.find(ST_STEP_END)
    return hashlib.sha256(data[:cut] if cut >= 0 else data).hexdigest()[:16]


def traffic_from_profile(kernel_src):
    """DRAM bytes per launch of the chain kernel from the committed ncu summary, if its
    source (ops.cu up to the batched kernel) is the one the counters were taken on."""
    path = os.path.join(ROOT, "profiles", "ncu_st_step_horner_convdiff128.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        parts = line.split()
        if len(parts) >= 2 and parts[0].endswith(":"):
            vals[parts[0][:-1]] = parts[1]
    if vals.get("st_step_src_sha256_16") != st_step_source_hash(kernel_src):
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def load_peak():
    """(HBM GB/s, source): the measured copy bandwidth, else the 6.8 TB/s fallback."""
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        return float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def events_time(fn, reps, stream, flush=None):
    """Mean milliseconds of fn() over reps calls, CUDA events on `stream`
    around each call (after a flush of L2 when given), synchronised."""
    import torch
    ms = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms)


def chain_out_of_l2(pp, torch, degree=16, reps=5):
    """The stencil chain out of L2: q(A) x by pp_poly_apply on the 2D Laplacian
    8192^2 (vectors of 268 MB in FP32), Horner form, FP32 and double-word.
    Algorithmic bytes of one call: the FP64 input converted in and the result
    converted out ((8 + s) bytes per entry each way), the first step (2
    vectors) and deg - 1 Horner steps (3 vectors each), s = 4 (FP32) or 8."""
    peak, src = load_peak()
    dims = (8192, 8192)
    n = dims[0] * dims[1]
    stream = torch.cuda.current_stream()
    h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims, stream=stream)
    out = {"workload": "2D Laplacian 8192^2 (n=67108864), q(A) x by pp_poly_apply, Chebyshev degree %d "
                       "in Newton/Horner form" % degree, "peak": peak, "peak_source": src, "unit": "GB/s"}
    try:
        pp.pp_build_poly(h, degree)
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
        y = torch.empty_like(x)
        for name, prec, esz in (("f32", pp.PP_PREC_MIXED, 4), ("dw", pp.PP_PREC_DW, 8)):
            o = pp.pp_default_opts()
            o.precision = prec
            pp.pp_set_opts(h, o)
            for _ in range(2):
                pp.pp_poly_apply(h, x, y)
            ms = events_time(lambda: pp.pp_poly_apply(h, x, y), reps, stream)
            byt = ((2 + 3 * (degree - 1)) * esz + 2 * (8 + esz)) * n
            gbs = byt / (ms * 1e-3) / 1e9
            out[name] = {"achieved": gbs, "frac": gbs / peak, "us_per_step": 1e3 * ms / degree,
                         "bytes_per_call": byt, "ms_per_call": ms}
        del x, y
    finally:
        pp.pp_destroy(h)
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2401_06684_gb300 import build as ppbuild
    from paper_2401_06684_gb300 import pp
    import synth

    rank, ws, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(pp.LIB_PATH):
        if rank == 0 or ws == 1:
            ppbuild.build()
        if ws > 1:
            dist.barrier()
    stream = torch.cuda.current_stream()
    dims = args.dims
    n = args.n
    keep = []
    PREC = {"dw": pp.PP_PREC_DW, "f64": pp.PP_PREC_F64, "mixed": pp.PP_PREC_MIXED}

    def make_handle(degree):
        if args.kind == "convdiff3d7":
            hh = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5], stream=stream)
            pp.pp_build_poly(hh, degree)
        elif args.kind == "laplace2d5":
            hh = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims, stream=stream)
            pp.pp_build_poly(hh, degree)
        elif args.kind == "wilson4d":
            keep.append(torch.from_numpy(synth.wilson_links(dims, 1)).cuda())
            hh = pp.pp_create_stencil(pp.PP_WILSON4D_DHD, dims, [WILSON_M0], links=keep[-1],
                                      dtype=pp.PP_C128, stream=stream)
            pp.pp_build_poly(hh, degree)
        elif args.kind == "wilsonq2":  # Example 2: Q^2 with the chemical potential, q at Ritz values
            keep.append(torch.from_numpy(synth.wilson_links(dims, 1)).cuda())
            hh = pp.pp_create_stencil(pp.PP_WILSON4D_Q2, dims, [SIGN_MW, SIGN_MU], links=keep[-1],
                                      dtype=pp.PP_C128, stream=stream)
            pp.pp_build_poly(hh, degree, pp.PP_RITZ_LEJA)
        elif args.kind == "graphcsr":  # Example 3: non-Hermitian CSR, q at Ritz values
            rp, col, val = graph_csr(n)
            keep.extend(torch.from_numpy(a).cuda() for a in (rp, col, val))
            hh = pp.pp_create_csr(n, *keep[-3:], is_hermitian=False, stream=stream)
            pp.pp_build_poly(hh, degree, {"ritz": pp.PP_RITZ_LEJA, "harmonic": pp.PP_HARMONIC_RITZ,
                                          "lsq": pp.PP_LSQ_CONTOUR}[args.poly or "ritz"])
        else:  # 2D Laplacian in CSR: interval from the closed form of its eigenvalues
            rp, col, val = synth.stencil_csr("laplace2d5", dims)
            keep.extend(torch.from_numpy(a).cuda() for a in (rp, col, val))
            hh = pp.pp_create_csr(n, *keep[-3:], is_hermitian=True, stream=stream)
            lo = sum(2.0 - 2.0 * math.cos(math.pi / (N + 1)) for N in dims)
            hi = sum(2.0 - 2.0 * math.cos(N * math.pi / (N + 1)) for N in dims)
            pp.pp_build_poly(hh, degree, interval_ab=(lo, hi))
        return hh

    def opts_for(prec, profile=0):
        o = pp.pp_default_opts()
        o.precision = PREC[prec]
        if args.two_pass or args.workload == "laplace8192":  # O(n) basis memory: two-pass Lanczos
            o.two_pass = 1
        o.clenshaw = 1 if args.clenshaw else 0
        o.orth = {"cgs2": pp.PP_ORTH_CGS2, "dcgs2": pp.PP_ORTH_DCGS2}.get(args.orth, pp.PP_ORTH_AUTO)
        o.halo = 1 if args.halo else 0
        if args.kind == "graphcsr":  # Example 3 checks every 32/d iterations
            o.check_every = max(1, 32 // (args.degree + 1))
        if args.kind == "wilsonq2":  # Example 2 checks every 64/d iterations
            o.check_every = max(1, 64 // (args.degree + 1))
        o.profile = profile
        return o

    h = make_handle(args.degree)
    o = opts_for(args.prec)
    pp.pp_set_opts(h, o)
    if args.autotune:
        args.degree = pp.pp_autotune(h, args.tol, 64)
    vdt = torch.complex128 if args.complex else torch.float64
    esz = 16 if args.complex else 8

    def rhs_host(seed):
        if args.kind == "graphcsr":
            return synth.unit_vector(n, 4 + seed)
        return synth.spinor_field(dims, seed) if args.complex else synth.rhs(n, seed)

    b = torch.from_numpy(rhs_host(rank)).cuda()
    x = torch.empty(n, dtype=vdt, device="cuda")
    s2 = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    m_max = args.m_max

    def solve(hh=h, out=x, m=m_max):
        return pp.pp_apply(hh, args.func, b, out, m_max=m, tol=args.tol)

    # the clock sampler starts before the warm-up solves: its nvidia-smi start-up (NVML
    # initialisation) stays out of the timed steps, its samples still cover all of them
    clk = ClockSampler(local)
    for _ in range(args.warmup):
        st = solve()
        assert st.status == pp.PP_OK, st.as_dict()

    # ---- timed solves (they replay the library's captured segment graphs; no per-run events inside)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        st = solve()
        ev[i][1].record(stream)
        stats.append(st.as_dict())
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    step_ms = [a.elapsed_time(e) for a, e in ev]
    t_total = max_over_ranks(sum(step_ms) / 1e3, ws)
    value = replica_value(args.steps, ws, t_total)
    x_timed = x.cpu().numpy().copy()  # the result of the last timed solve

    # ---- the chain's roofline: one untimed solve with CUDA events around every run of operator launches
    pp.pp_set_opts(h, opts_for(args.prec, profile=1))
    flush.zero_()
    pst = solve().as_dict()
    pp.pp_set_opts(h, o)
    chain_ms, chain_bytes, chain_launches = pst["chain_ms"], pst["chain_bytes"], pst["chain_launches"]
    # where the profiled solve's time goes (direct launches with events: slower than the timed,
    # graph-replayed solves; "other" = start vector, reconstruction, launch gaps and the host
    # round trip of every stopping check)
    breakdown = {"profiled_solve_ms": pst["ms_total"], "chain_ms": chain_ms, "orth_ms": pst["orth_ms"],
                 "small_solve_ms": pst["small_ms"],
                 "other_ms": pst["ms_total"] - chain_ms - pst["orth_ms"] - pst["small_ms"],
                 "checks": pst["checks"]}
    achieved = chain_bytes / (chain_ms / 1e3) / 1e9 if chain_ms > 0 else None
    peak, peak_src = load_peak()
    traffic = (traffic_from_profile(os.path.join(ROOT, "paper_2401_06684_gb300", "csrc", "ops.cu"))
               if args.workload == "convdiff128" and not args.clenshaw else None)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    bh = torch.from_numpy(rhs_host(rank)).pin_memory()
    xh = torch.empty(n, dtype=vdt).pin_memory()
    e2e_t = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pp.pp_apply_host(h, args.func, bh.data_ptr(), xh.data_ptr(), m_max=m_max, tol=args.tol)
        if i > 0:
            e2e_t.append(time.perf_counter() - t0)
    e2e_val = replica_value(len(e2e_t), ws, max_over_ranks(sum(e2e_t), ws))

    # ---- accuracy, outside the timed region.  The identity's reference (A b for SQRT, b for
    # INVSQRT / SIGN) comes from a double-word (FP64-grade) operator application, never from
    # the FP32 one of mixed precision.
    if args.func == pp.PP_SIGN:
        ref_id, id_name = b, "identity_sign_sign_vs_b"
        pp.pp_apply(h, pp.PP_SIGN, x, s2, m_max=m_max, tol=args.tol)
    elif args.func > 0:
        ref_id, id_name = torch.empty_like(x), "identity_sqrt_sqrt_vs_Ab"
        pp.pp_set_opts(h, opts_for("dw"))
        pp.pp_op_apply(h, b, ref_id)
        pp.pp_set_opts(h, o)
        pp.pp_apply(h, pp.PP_SQRT, x, s2, m_max=m_max, tol=args.tol)
    else:
        ref_id, id_name = b, "identity_sqrt_of_invsqrt_vs_b"
        pp.pp_apply(h, pp.PP_SQRT, x, s2, m_max=m_max, tol=args.tol)
    torch.cuda.synchronize()
    ident = float(torch.linalg.norm(s2 - ref_id) / torch.linalg.norm(ref_id))

    # ---- companions in the other arithmetics on the same handle and b, and the in-GPU
    # baselines: plain unpreconditioned Arnoldi / Lanczos (degree 0) in FP64 and double-word
    comp = {}
    if not args.no_companions and rank == 0:
        for prec in ("dw", "f64"):
            if prec == args.prec:
                continue
            pp.pp_set_opts(h, opts_for(prec))
            for _ in range(2):
                solve(out=s2)
            reps = max(3, min(args.steps, 10))
            ms = events_time(lambda: solve(out=s2), reps, stream, flush)
            stc = solve(out=s2)
            torch.cuda.synchronize()
            comp[prec] = {"value": 1e3 / ms, "unit": "solves/s", "ms_per_solve": ms, "solves_timed": reps,
                          "iters": stc.iters, "mvms": stc.mvms, "status": pp.pp_strerror(stc.status),
                          "x": s2.cpu().numpy().copy()}
        pp.pp_set_opts(h, o)
    plain = {}
    if not args.no_plain and rank == 0:
        hp = make_handle(0)
        for prec in ("f64", "dw"):
            pp.pp_set_opts(hp, opts_for(prec))
            st0 = pp.pp_apply(hp, args.func, b, s2, m_max=args.plain_m_max, tol=args.tol)
            torch.cuda.synchronize()
            # a run that hit m_max without meeting tol is no solve: no value
            plain[prec] = {"value": 1e3 / st0.ms_total if st0.status == pp.PP_OK else None, "unit": "solves/s",
                           "iters": st0.iters, "m_max": args.plain_m_max, "status": pp.pp_strerror(st0.status),
                           "x": s2.cpu().numpy().copy()}
        pp.pp_destroy(hp)

    # ---- the stencil chain out of L2 (8192^2), and the 128^3 chain counted in DRAM bytes
    out_l2 = None
    if not args.no_out_of_l2 and rank == 0 and args.kind in ("convdiff3d7", "laplace2d5"):
        out_l2 = chain_out_of_l2(pp, torch)

    m_full = stats[-1]["iters"]
    pp.pp_destroy(h)
    del flush

    # ---- host work: the oracle's whole solve (cpu_baseline) and its x* (accuracy)
    cpu, ref, ref_how = None, None, "not computed"
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, run = cpu_sample(args, m_full)
        if not args.no_oracle_err:
            ref, ref_how = oracle_reference(args, rank, run)
    elif rank == 0 and not args.no_oracle_err:
        ref, ref_how = oracle_reference(args, rank, None)

    def err_or_none(xv):
        return rel_err(xv, ref) if ref is not None else None

    if rank == 0:
        for d in list(comp.values()) + list(plain.values()):
            d["rel_err_vs_oracle"] = err_or_none(d.pop("x"))
        mixed_dtype = args.prec == "mixed" and stats[-1]["switch_iter"] >= 0
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "ms_per_step_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)],
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32x2-dw+f32" if mixed_dtype else {"dw": "f32x2-dw", "f64": "f64", "mixed": "f32x2-dw"}[args.prec]),
            "precision": ("double-word start, FP32 chain/basis/updates after switch_iter, FP64 coefficients and "
                          "small solve" if mixed_dtype else
                          "double-word FP32 pairs throughout (the switch rule never allowed FP32)" if args.prec == "mixed"
                          else {"dw": "double-word FP32 pairs (FP64-grade)", "f64": "IEEE FP64"}[args.prec]),
            "data": "synthetic (b ~ N(0,1), seed = rank)", "config": config(args, ws),
            "accuracy": {"rel_err_vs_oracle": err_or_none(x_timed), "oracle": ref_how,
                         "target": accuracy_target(args),
                         id_name: ident, "est_err_last": stats[-1]["est_err"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": "%s (operator + %s update)" % (
                             {"graphcsr": "csr_step", "laplace2d5csr": "csr_step", "wilson4d": "wilson_step",
                              "wilsonq2": "wilson_q_step"}.get(
                                 args.kind, "st_step"), "Clenshaw" if args.clenshaw else "Horner"),
                         "peak_source": peak_src,
                         "timing": "CUDA events around each run of consecutive operator launches "
                                   "(one q(A) or one A product) in one untimed solve after the timed ones "
                                   "(those replay the library's CUDA graphs of the steps between stopping "
                                   "checks)",
                         "launches": chain_launches,
                         "bytes_per_launch": chain_bytes / max(chain_launches, 1),
                         "dram_frac": (traffic * chain_launches / (chain_ms / 1e3) / 1e9 / peak
                                       if traffic and chain_ms > 0 else None),
                         "out_of_l2": out_l2,
                         **({"note": "the double-word Wilson kernel is bound by the FP32 pipe, not HBM: FMA "
                                     "pipe 51 % active, issue 56 %, DRAM 11-19 % busy (ncu, "
                                     "profiles/ncu_wilson_q_step_dw_sign16x32.txt); frac is the HBM fraction "
                                     "of the metric"}
                            if args.kind in ("wilson4d", "wilsonq2") and args.prec != "f64" else {})},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": esz * n,
                    "d2h_bytes_per_step": esz * n},
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "clocks": clocks,
            "switch_iter": stats[-1]["switch_iter"],
            "iters": m_full, "mvms": stats[-1]["mvms"], "wall_s": wall,
            "breakdown": breakdown,
            "companions": comp or None,
            "plain_gpu": plain or None,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_batch(args):
    """The batched workload: one pp_apply_batch call per step."""
    import torch
    from paper_2401_06684_gb300 import build as ppbuild
    from paper_2401_06684_gb300 import pp
    import synth

    rank, ws, local = dist_env()
    torch.cuda.set_device(local)
    if not os.path.exists(pp.LIB_PATH):
        ppbuild.build()
    stream = torch.cuda.current_stream()
    probs = synth.batch_problems(64, seed=2 + 100 * rank)
    kinds = {"laplace2d5": pp.PP_LAPLACE2D5, "laplace3d7": pp.PP_LAPLACE3D7,
             "convdiff3d7": pp.PP_CONVDIFF3D7_UPWIND}
    prec = {"dw": pp.PP_PREC_DW, "f64": pp.PP_PREC_F64, "mixed": pp.PP_PREC_MIXED}[args.prec]
    hs, bs, xs, bh, xh, degs = [], [], [], [], [], []
    for i, p in enumerate(probs):
        h = pp.pp_create_stencil(kinds[p["kind"]], p["dims"], [0.5] if p["kind"] == "convdiff3d7" else None,
                                 stream=stream)
        o = pp.pp_default_opts()
        o.precision = prec
        pp.pp_set_opts(h, o)
        degs.append(pp.pp_autotune(h, args.tol, 64))
        n = 1
        for d in p["dims"]:
            n *= d
        B = synth.rhs(n, 1000 + i, nrhs=p["nrhs"]) if p["nrhs"] > 1 else synth.rhs(n, 1000 + i)[None, :]
        hs.append(h)
        bh.append(torch.from_numpy(B.reshape(-1)).pin_memory())
        xh.append(torch.empty(B.size, dtype=torch.float64).pin_memory())
        bs.append(bh[-1].cuda())
        xs.append(torch.empty(B.size, dtype=torch.float64, device="cuda"))
    fs = [p["f"] for p in probs]
    nr = [p["nrhs"] for p in probs]
    nsolves = sum(nr)
    rows = sum(int(b.numel()) for b in bs)

    # one batch plan (allocations, tables and, after the first solve, the captured segment
    # graphs of every group), then one pp_batch_apply per step
    plan = pp.pp_batch_create(hs, fs, nrhs=nr, m_max=args.m_max, stream=stream)

    def step():
        return pp.pp_batch_apply(plan, bs, xs, tol=args.tol)

    clk = ClockSampler(local)  # started before the warm-up (see run_ours)
    for _ in range(args.warmup):
        st = step()
        assert all(q.status == pp.PP_OK for q in st)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    stats = None
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        stats = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_total = sum(a.elapsed_time(e) for a, e in ev) / 1e3
    value = args.steps * nsolves / t_total
    # operator-chain profiling in one more (untimed) step: CUDA events around
    # every run of batched stencil launches, the groups run one after another
    o = pp.pp_default_opts()
    o.precision = prec
    o.profile = 1
    pp.pp_set_opts(hs[0], o)
    flush.zero_()
    stats = step()
    torch.cuda.synchronize()
    o.profile = 0
    pp.pp_set_opts(hs[0], o)
    peak, peak_src = load_peak()
    cb, cms, cl = stats[0].chain_bytes, stats[0].chain_ms, stats[0].chain_launches
    # (the profiled step launched its kernels directly, so their events bracket them)
    achieved = cb / (cms / 1e3) / 1e9 if cms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": "bst_step (batched operator + Horner update, one step of every process)",
                "peak_source": peak_src,
                "timing": "CUDA events around each run of batched operator launches in one untimed step after "
                          "the timed ones, groups run one after another",
                "launches": cl, "bytes_per_launch": cb / max(cl, 1)}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_sample_batch(args, probs)
    # end to end: pinned host b in, batch, host x out
    e2e_t = []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(len(bs)):
            bs[q].copy_(bh[q], non_blocking=True)
        step()
        for q in range(len(xs)):
            xh[q].copy_(xs[q], non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    iters = [q.iters for q in stats]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"dw": "f32x2-dw", "f64": "f64", "mixed": "f32x2-dw+f32"}[args.prec],
        "data": "synthetic (problem list seed 2, b ~ N(0,1) seed 1000 + i)",
        "config": {"workload": args.desc, "problems": len(probs), "right_hand_sides": nsolves,
                   "rows_total": rows, "tol": args.tol, "parallelism": f"replicas{ws}",
                   "l2": "flushed between timed steps (256 MB write)"},
        "autotuned_degrees": sorted(set(degs)), "iters_min_max": [min(iters), max(iters)],
        "gpu_launches": int(stats[0].launches), "e2e": {"value": args.steps * nsolves / sum(e2e_t),
                                                         "unit": "solves/s", "h2d_bytes_per_step": 8 * rows,
                                                         "d2h_bytes_per_step": 8 * rows},
        "clocks": clocks, "roofline": roofline, "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    pp.pp_batch_destroy(plan)
    for h in hs:
        pp.pp_destroy(h)


def run_probe(args):
    """Per-launch timing of the operator kernels on the workload's stencil
    (not a bench line): q(A) v by pp_poly_apply (one launch per step) in FP32
    and double-word, Horner and Clenshaw, one operator application in each
    arithmetic, and device copies of 8 MB / 32 MB / 1 GB for scale.  The
    command an ncu capture of the stencil step kernel runs."""
    import torch
    from paper_2401_06684_gb300 import pp
    import synth
    if args.kind not in ("convdiff3d7", "laplace2d5"):
        raise SystemExit("--probe: stencil workloads only")
    dims = tuple(args.dims)
    n = int(np.prod(dims))
    if args.kind == "convdiff3d7":
        h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5])
    else:
        h = pp.pp_create_stencil(pp.PP_LAPLACE2D5, dims)
    pp.pp_build_poly(h, args.degree)
    x = torch.from_numpy(synth.rhs(n, 1)).cuda()
    y = torch.empty_like(x)
    reps = args.steps

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return 1e3 * e0.elapsed_time(e1) / reps

    peak, src = load_peak()
    res = {"peak_GBs": peak, "peak_source": src}
    for name, prec, esz in (("f32", pp.PP_PREC_MIXED, 4), ("dw", pp.PP_PREC_DW, 8)):
        for scheme in ("horner", "clenshaw"):
            o = pp.pp_default_opts()
            o.precision = prec
            o.clenshaw = int(scheme == "clenshaw")
            pp.pp_set_opts(h, o)
            k = max(args.degree, 1)
            us = timed(lambda: pp.pp_poly_apply(h, x, y))
            # algorithmic bytes of one q(A) x by pp_poly_apply: the FP64 input
            # converted in and the result out (8 + s bytes per entry each way),
            # then the chain: first step 2 vectors, Horner steps 3, Clenshaw
            # steps 3 (the second) and 4 (the others)
            chain = 2 + (3 * (k - 1) if scheme == "horner" else (3 + 4 * (k - 2) if k >= 2 else 0))
            byt = (chain * esz + 2 * (8 + esz)) * n
            res[f"{name}_{scheme}_us_per_step"] = us / k
            res[f"{name}_{scheme}_GBs"] = byt / (us * 1e-6) / 1e9
            res[f"{name}_{scheme}_frac"] = byt / (us * 1e-6) / 1e9 / peak
    for name, prec in (("f32", pp.PP_PREC_MIXED), ("dw", pp.PP_PREC_DW), ("f64", pp.PP_PREC_F64)):
        o = pp.pp_default_opts()
        o.precision = prec
        pp.pp_set_opts(h, o)
        res[f"{name}_op_apply_us"] = timed(lambda: pp.pp_op_apply(h, x, y))
    for mb in (8, 32, 1024):
        a = torch.empty(mb << 18, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        us = timed(lambda: b.copy_(a))
        res[f"copy_{mb}MB_us"] = us
        res[f"copy_{mb}MB_GBs"] = 2 * (mb << 20) / (us * 1e-6) / 1e9
    pp.pp_destroy(h)
    print(json.dumps({"probe": res, "workload": args.desc, "degree": args.degree, "reps": reps}), flush=True)


def main():
    args = parse()
    if args.probe:
        run_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.kind == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
