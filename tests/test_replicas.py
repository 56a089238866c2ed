"""The multi-GPU form is N independent replicas (one graph per rank, no
collective on the data path). Its host side runs here on CPU with gloo,
world size 2: each rank draws its own graph of the same size, timings are
the maximum over ranks, the job rate is all ranks' edges over that time;
and under torchrun the reference arm prints exactly one line, from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import hashlib

    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    w = bench.make_workload("tiny", 1.0, rank)
    h = hashlib.sha256(w.src.tobytes() + w.dst.tobytes() + w.t.tobytes()).hexdigest()
    seen = [None] * world
    dist.all_gather_object(seen, (w.n_edges, h))
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, seen, slowest))


def test_two_replicas_on_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seen, slowest in out:
        (e0, h0), (e1, h1) = seen
        assert e0 == e1 and h0 != h1          # same size, own seed per rank
        assert slowest == 20.0                # max over ranks
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(2, 1000, 0.5) == 4000.0
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "tiny", "--cpu-sample-minutes", "60"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0


def test_reference_sample_shrinks_with_step_count():
    """The reference arm keeps its whole run to a few minutes of one core:
    unless a window is given, more steps take a shorter window each."""
    import argparse
    import bench
    for wl in ("hub", "mid"):
        win = [bench.reference_sample_minutes(argparse.Namespace(cpu_sample_minutes=None, steps=s, warmup=3), wl)
               for s in (5, 10, 20, 50)]
        assert win == sorted(win, reverse=True) and win[0] == bench.CPU_SAMPLE_MINUTES[wl]
        assert win[-1] < win[0]
    given = argparse.Namespace(cpu_sample_minutes=42.0, steps=100, warmup=3)
    assert bench.reference_sample_minutes(given, "hub") == 42.0
