"""Multi-GPU path of the bench on the host: ranks are independent replicas
(no collective on the data path); the job's time is the slowest rank's, taken
by an all-reduce MAX, and only rank 0 prints.  world_size 2 over gloo, CPU only."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    local = [1.5, 2.5][rank]  # per-rank timed seconds
    t = bench.max_over_ranks(local, ws)
    out[rank] = (t, bench.replica_value(10, ws, t))
    dist.destroy_process_group()


def test_max_over_ranks_and_value():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    for rank in range(ws):
        t, v = out[rank]
        assert t == 2.5                 # the slowest rank sets the time
        assert v == ws * 10 / 2.5       # units of all ranks over that time


def test_reference_arm_only_rank0_prints():
    # --impl reference under torchrun: rank 1 exits 0 without work and prints nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.replica_value(30, 1, 0.5) == 60.0
    # rank r solves right-hand side seed r: replicas do distinct work
    import synth
    assert not (synth.rhs(100, 0) == synth.rhs(100, 1)).all()
