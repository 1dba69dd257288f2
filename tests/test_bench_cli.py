"""The bench's command line and configuration (host only): every workload
parses with its defaults, the headline workload is the 128^3
convection-diffusion square root with delayed reorthogonalization in mixed
precision, --orth applies to the Arnoldi workloads only, and the oracle runs
CGS2 for a DCGS2 workload (the same basis in exact arithmetic)."""
import sys

import pytest

import bench


def parse(argv, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench.parse()


def test_every_workload_parses(monkeypatch):
    for w in bench.WORKLOADS:
        a = parse(["--workload", w], monkeypatch)
        assert a.m_max == {"sign32x64": 200, "convdiff256": 100}.get(w, 1000)
        if a.kind == "batch":  # the batch runner writes its own configuration
            continue
        cfg = bench.config(a, 1)
        assert cfg["workload"] and cfg["orth"] == a.orth and cfg["tol"] == a.tol


def test_headline_defaults(monkeypatch):
    a = parse([], monkeypatch)
    assert a.workload == "convdiff128" and a.dims == (128, 128, 128) and a.func == 1
    assert a.degree == 16 and a.tol == 1e-10 and a.prec == "mixed" and a.orth == "dcgs2"
    assert a.steps >= 1 and a.warmup >= 3
    assert bench.config(a, 1)["fp32_stencil_steps"] == "one per launch"


def test_orth_option(monkeypatch):
    assert parse(["--orth", "cgs2"], monkeypatch).orth == "cgs2"
    assert parse(["--workload", "graph282k", "--orth", "dcgs2"], monkeypatch).orth == "dcgs2"
    with pytest.raises(SystemExit):
        parse(["--workload", "laplace2048", "--orth", "dcgs2"], monkeypatch)  # a Lanczos workload
