"""The bench's multi-rank logic on CPU: two gloo ranks (127.0.0.1).

Each rank times its own replica of the workload (weak scaling); the job's
time is the slowest rank's, and its value counts the frames of every rank.
The reference arm runs on rank 0 alone: other ranks print nothing and exit 0.
"""
import json
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


def _rank(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        got = bench.whole_job(ms, frames_per_step=1000, steps=4, world=world, dev=torch.device("cpu"))
        with open(out_path, "w") as f:
            json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    outs = [str(tmp_path / f"r{r}.json") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for o in outs:
        ms, value = json.load(open(o))
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_whole_job_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job(8.0, 500, 2, 1, None)
    assert ms == 8.0 and value == pytest.approx(500 * 2 / 0.008)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
