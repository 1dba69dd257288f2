"""A process pool for oracle solves in the GPU tests (test infrastructure).

Oracle solves of many independent problems run in parallel worker
processes, each with a few OpenMP threads for the oracle's CSR product.
The pool uses the "spawn" start method: a process forked from one that has
initialised CUDA can hang.
"""
import multiprocessing as mp
import os


def _init(threads):
    os.environ["OMP_NUM_THREADS"] = str(threads)


def convdiff_solve(job):
    """x* of one convection-diffusion process: the oracle's Algorithm 1
    (Chebyshev degree 16, CGS2, left) to a stopping estimate of 1e-12."""
    dims, b, power = job
    from oracle import chebyshev as cheb, krylov, operators as ops, spmv
    A = ops.convdiff(dims, 0.5)
    a, b_ = ops.convdiff_interval(dims, 0.5)
    r = krylov.pp_arnoldi(spmv.CsrMv(A), b, power, cheb.interp_coeffs(a, b_, 17), (a, b_), side="left",
                          m_max=300, tol=1e-12, k_chk=3, orth="cgs2")
    if not r["converged"]:
        raise RuntimeError("oracle solve did not converge")
    return r["x"]


def map_spawn(fn, jobs, workers=None, threads=2):
    """[fn(j) for j in jobs] in spawned worker processes."""
    cores = os.cpu_count() or 2
    workers = workers or max(1, cores // threads)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_init, initargs=(threads,)) as pool:
        return pool.map(fn, jobs, chunksize=1)
