"""Host-side work order of the persistent kernels (no GPU).

The kernels walk the tile list on a static schedule: worker w takes units
w, w + W, w + 2W, ... of `unit` tiles (two for CTA pairs, whose pair of MMAs
waits for the longer tile).  The balancer permutes the list; these tests
check that it is a permutation that keeps the lone tile of an odd count in
the last position, and that its longest worker is no longer than in clip
order, on the batch shapes the kernels run.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_01009_gb300", "csrc")
TILE = 128
FIXED = 40  # fixed per-tile cost in frames used by the balancer


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = str(tmp_path_factory.mktemp("sched") / "sched_harness")
    cmd = [cxx, "-std=c++17", "-O2", "-I", cuda_inc, "-x", "c++",
           os.path.join(ROOT, "tests", "sched_harness.cpp"),
           os.path.join(CSRC, "melt_schedule.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "cuda_runtime.h" in r.stderr:
            pytest.skip("CUDA headers not found")
        raise RuntimeError(r.stderr)
    return exe


def run(exe, cases):
    """cases: list of (frames list, unit, W) -> list of index orders."""
    text = "".join(f"{len(f)} {u} {w}\n" + " ".join(map(str, f)) + "\n" for f, u, w in cases)
    r = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
    return [np.array(list(map(int, line.split())), dtype=np.int64) for line in r.stdout.splitlines()]


def clip_tiles(n_frames_per_clip):
    out = []
    for T in n_frames_per_clip:
        out += [min(TILE, T - t0) for t0 in range(0, T, TILE)]
    return out


def makespan(frames, order, unit, W):
    f = np.asarray(frames)[order]
    n = len(f)
    N = (n + unit - 1) // unit
    load = np.zeros(W, dtype=np.int64)
    for u in range(N):
        load[u % W] += f[u * unit:(u + 1) * unit].max() + FIXED
    return int(load.max())


def check_order(frames, order, unit):
    n = len(frames)
    assert sorted(order.tolist()) == list(range(n))
    if unit == 2:
        f = np.asarray(frames)[order]
        # members of a pair come from adjacent places in the length ranking
        ranks = np.empty(n, dtype=np.int64)
        ranks[np.argsort(-np.asarray(frames), kind="stable")] = np.arange(n)
        r = ranks[order]
        for q in range(n // 2):
            assert abs(r[2 * q] - r[2 * q + 1]) == 1
        assert f.max() <= TILE


def test_thirty_second_clips_lose_a_round(harness):
    # 64 clips x 2998 frames: 1536 tiles, 768 pairs over 76 clusters.  In clip
    # order 8 clusters run 11 pairs of full cost; balanced, no cluster runs
    # more than 10 full-tile units of work.
    frames = clip_tiles([2998] * 64)
    ident = np.arange(len(frames))
    (order,) = run(harness, [(frames, 2, 76)])
    check_order(frames, order, 2)
    assert makespan(frames, ident, 2, 76) == 11 * (TILE + FIXED)
    assert makespan(frames, order, 2, 76) == 10 * (TILE + FIXED)


@pytest.mark.parametrize("unit,W", [(1, 152), (2, 76), (2, 5), (1, 1), (2, 1)])
def test_random_batches(harness, unit, W):
    rng = np.random.default_rng(1234 + unit * 1000 + W)
    cases = []
    for _ in range(40):
        batch = int(rng.integers(1, 400))
        T = rng.integers(1, 4000, size=batch)
        cases.append((clip_tiles(T.tolist()), unit, W))
    for (frames, u, w), order in zip(cases, run(harness, cases)):
        check_order(frames, order, u)
        ms = makespan(frames, order, u, w)
        assert ms <= makespan(frames, np.arange(len(frames)), u, w)
        n_units = (len(frames) + u - 1) // u
        per_worker = -(-n_units // w)
        assert ms <= per_worker * (TILE + FIXED)


@pytest.mark.parametrize("n", [1, 2, 3, 151, 152, 153, 305])
def test_odd_counts_keep_the_lone_tile_last(harness, n):
    rng = np.random.default_rng(n)
    frames = rng.integers(1, TILE + 1, size=n).tolist()
    (order,) = run(harness, [(frames, 2, 76)])
    check_order(frames, order, 2)
    if n % 2:
        # the lone tile (last position, a pair of its own) is a shortest tile
        assert frames[order[-1]] == min(frames)


def test_oversized_schedule_is_left_alone(harness):
    frames = clip_tiles([300, 5000, 129])
    (order,) = run(harness, [(frames, 2, 4096)])
    assert order.tolist() == list(range(len(frames)))
