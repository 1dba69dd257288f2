#!/usr/bin/env python3
"""Throughput of polynomially preconditioned f(A)b on GB300.

One step = one complete solve x = A^{1/2} b (Algorithm 1 with A^{1/2} b =
A^{-1/2}(A b)) of the 3D upwind convection-diffusion operator on a 128^3 grid
(n = 2,097,152, c*h = 0.5, non-Hermitian, so Arnoldi with CGS2), Chebyshev q
of degree 16 on the exact spectral interval, stopping estimate < 1e-10.  The
metric is solves per second over all ranks; ranks solve independent
right-hand sides (seed 0 + rank), no collective on the data path.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "f(A)b solves/sec and SpMV-chain HBM GB/s (% roofline) at 1e-8 rel err vs FP64 oracle"
WORKLOAD = "3D convection-diffusion 128^3 upwind 7-point (n=2097152, c*h=0.5), f=A^(1/2), Arnoldi CGS2"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--degree", type=int, default=16)
    p.add_argument("--prec", default="dw", choices=["dw", "f64"])
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--cpu-iters", type=int, default=3)
    p.add_argument("--m-max", type=int, default=400)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def config(args, ws):
    return {"workload": WORKLOAD, "grid": [args.grid] * 3, "n": args.grid ** 3, "ch": 0.5,
            "func": "sqrt", "poly": "chebyshev", "degree": args.degree, "side": "left",
            "orth": "cgs2", "tol": args.tol, "rhs_per_rank": 1, "parallelism": f"replicas{ws}",
            "l2": "flushed between timed steps (256 MB write)"}


# ---------------------------------------------------------------- oracle (CPU)

def oracle_timed(grid, degree, m_max, tol, seed=0):
    """Run the FP64 oracle (Algorithm 1, as it stands) and time its set-up and iterations.

    Returns (result, setup seconds, list of per-iteration seconds)."""
    from oracle import chebyshev as cheb, krylov, operators as ops
    import synth
    dims = (grid,) * 3
    A = ops.convdiff(dims, 0.5)
    a, b = ops.convdiff_interval(dims, 0.5)
    c = cheb.interp_coeffs(a, b, degree + 1)
    rhs = synth.rhs(A.shape[0], seed)
    stamps = []
    t0 = time.perf_counter()
    r = krylov.pp_arnoldi(A.dot, rhs, 0.5, c, (a, b), side="left", m_max=m_max, tol=tol,
                          k_chk=max(1, 64 // (degree + 1)), hermitian=False, orth="cgs2",
                          on_iter=lambda j: stamps.append(time.perf_counter()))
    t_end = time.perf_counter()
    setup = stamps[0] - t0
    iters = [b_ - a_ for a_, b_ in zip(stamps[:-1], stamps[1:])]
    r["tail_s"] = t_end - stamps[-1]
    return r, setup, iters


def cpu_sample(args, m_full):
    """The oracle on the full workload for a few iterations, extrapolated to m_full iterations."""
    k = max(1, args.cpu_iters)
    r, setup, iters = oracle_timed(args.grid, args.degree, k, 0.0)
    t_iter = statistics.mean(iters)
    t_solve = setup + m_full * t_iter
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle Algorithm 1 (numpy/scipy FP64; SpMV single-threaded, OpenBLAS for the "
                      f"Gram-Schmidt products) run for {k} iterations on the full workload: set-up "
                      f"{setup:.2f}s + {t_iter:.2f}s/iteration, extrapolated to the {m_full} iterations "
                      f"of a solve = {t_solve:.1f}s"}


def run_reference(args):
    rank, ws, _ = dist_env()
    if rank != 0:
        return
    # Steps are oracle iterations on the full workload; full solves run until
    # warmup + steps iterations have been seen.  value = 1 / (set-up + m * mean
    # iteration time), m = the oracle's own iteration count.
    need = args.warmup + args.steps
    setups, iters, m = [], [], None
    while len(iters) < need:
        r, setup, its = oracle_timed(args.grid, args.degree, 400, args.tol)
        setups.append(setup)
        iters += its
        m = r["iters"]
    timed = iters[args.warmup:need]
    t_solve = statistics.mean(setups) + m * statistics.mean(timed)
    value = 1.0 / t_solve
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_solve,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (b ~ N(0,1), seed 0)", "config": config(args, 1),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} timed oracle iterations (after {args.warmup} warm-up "
                                       f"iterations) of full solves of this workload; a solve is set-up + "
                                       f"{m} iterations = {t_solve:.1f}s"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_iters": m}
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


def traffic_from_profile(kernel_src):
    """DRAM bytes per launch of the chain kernel from the committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "ncu_st3d_step_convdiff128.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(path):
        parts = line.split()
        if len(parts) >= 2 and parts[0].endswith(":"):
            vals[parts[0][:-1]] = parts[1]
    if vals.get("ops_cu_sha256_16") != h:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


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
    dims = (args.grid,) * 3
    n = args.grid ** 3
    h = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5], stream=stream)
    pp.pp_build_poly(h, args.degree)
    o = pp.pp_default_opts()
    o.precision = pp.PP_PREC_DW if args.prec == "dw" else pp.PP_PREC_F64
    pp.pp_set_opts(h, o)
    b = torch.from_numpy(synth.rhs(n, rank)).cuda()
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    m_max = args.m_max

    def solve():
        return pp.pp_apply(h, pp.PP_SQRT, b, x, m_max=m_max, tol=args.tol)

    for _ in range(args.warmup):
        st = solve()
        assert st.status == pp.PP_OK, st.as_dict()
    # accuracy of this configuration: (A^{1/2})^2 b = A b, outside the timed region
    s2 = torch.empty_like(x)
    ab = torch.empty_like(x)
    pp.pp_op_apply(h, b, ab)
    solve()
    pp.pp_apply(h, pp.PP_SQRT, x, s2, m_max=m_max, tol=args.tol)
    torch.cuda.synchronize()
    ident = float(torch.linalg.norm(s2 - ab) / torch.linalg.norm(ab))

    o.profile = 1
    pp.pp_set_opts(h, o)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    clk = ClockSampler(local)
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
    t_total = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([t_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
    o.profile = 0
    pp.pp_set_opts(h, o)
    value = ws * args.steps / t_total
    chain_ms = sum(s["chain_ms"] for s in stats)
    chain_bytes = sum(s["chain_bytes"] for s in stats)
    chain_launches = sum(s["chain_launches"] for s in stats)
    achieved = chain_bytes / (chain_ms / 1e3) / 1e9 if chain_ms > 0 else None
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_2401_06684_gb300", "csrc", "ops.cu"))

    # end to end through the C ABI with host buffers (copies inside the timed region)
    bh = torch.from_numpy(synth.rhs(n, rank)).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_t = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pp.pp_apply_host(h, pp.PP_SQRT, bh.data_ptr(), xh.data_ptr(), m_max=m_max, tol=args.tol)
        if i > 0:
            e2e_t.append(time.perf_counter() - t0)
    e2e_val = ws * len(e2e_t) / sum(e2e_t)
    if ws > 1:
        t = torch.tensor([sum(e2e_t)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_val = ws * len(e2e_t) / float(t.item())

    # in-GPU baseline: plain unpreconditioned Arnoldi (degree 0) in FP64 on the same problem
    plain = None
    if not args.no_plain and rank == 0:
        hp = pp.pp_create_stencil(pp.PP_CONVDIFF3D7_UPWIND, dims, [0.5], stream=stream)
        pp.pp_build_poly(hp, 0)
        st0 = pp.pp_apply(hp, pp.PP_SQRT, b, s2, m_max=1000, tol=args.tol)
        torch.cuda.synchronize()
        err0 = float(torch.linalg.norm(s2 - x) / torch.linalg.norm(x))
        plain = {"value": 1e3 / st0.ms_total, "unit": "solves/s", "iters": st0.iters, "prec": "f64",
                 "status": pp.pp_strerror(st0.status), "rel_diff_vs_preconditioned": err0}
        pp.pp_destroy(hp)

    m_full = stats[-1]["iters"]
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(args, m_full)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2-dw" if args.prec == "dw" else "f64",
            "data": "synthetic (b ~ N(0,1), seed = rank)", "config": config(args, ws),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": "st3d_step (operator + Clenshaw update)", "peak_source": peak_src,
                         "timing": "CUDA events around each run of consecutive operator launches "
                                   "(one q(A) or one A product) during the timed steps",
                         "launches": chain_launches,
                         "bytes_per_launch": chain_bytes / max(chain_launches, 1)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "clocks": clocks,
            "accuracy": {"identity_sqrt_sqrt_vs_Ab": ident, "est_err_last": stats[-1]["est_err"]},
            "iters": m_full, "mvms": stats[-1]["mvms"], "wall_s": wall,
            "plain_arnoldi_gpu": plain,
        }
        print(json.dumps(line), flush=True)
    pp.pp_destroy(h)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
