"""The N > 1 host path of bench.py on CPU: two gloo ranks (world_size 2).

The single-system workloads run as replicas (no data-path collective); the
only exchange is the timing reduction: every rank takes the slowest rank's
step time, and the job's rate is world systems per that time.  The reference
arm prints from rank 0 only.
"""
import importlib.util
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        ms = bench.max_over_ranks(10.0 + 3.0 * rank, dist, "cpu")
        out[rank] = (ms, bench.whole_job_gflops(world, 2.0e9, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, gf = out[0]
    assert ms == 13.0
    assert abs(gf - 2 * 2.0e9 / 13.0e-3 / 1e9) < 1e-9


def test_single_rank_needs_no_collective():
    bench = _bench()
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.whole_job_gflops(1, 1.0e9, 1.0) == 1000.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
