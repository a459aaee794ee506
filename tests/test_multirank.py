"""The multi-rank (replicas) path of bench.py on the CPU: two gloo ranks on
127.0.0.1. The whole-job value counts every rank's iterations over the
slowest rank's time; the reference arm runs on rank 0 only."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 200.0 + 10.0 * rank, steps=10, k=100,
                                         world=world, dist=dist, device="cpu")
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_all_iterations():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1]                       # every rank agrees
    value, e2e, job_ms, job_e2e = res[0]
    assert job_ms == 150.0 and job_e2e == 210.0   # max over ranks
    assert value == pytest.approx(2 * 10 * 100 / 0.150)
    assert e2e == pytest.approx(2 * 10 * 100 / 0.210)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, e2e, job_ms, _ = bench.aggregate_over_ranks(50.0, 60.0, steps=5, k=20, world=1)
    assert job_ms == 50.0 and value == pytest.approx(5 * 20 / 0.05)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""                 # only rank 0 prints the line
