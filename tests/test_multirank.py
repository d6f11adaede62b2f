"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The bench runs one independent replica per rank (the path is data-parallel
over independent domains, no collective on the data path): the job's time is
the slowest rank's, and its throughput counts every rank's cells.  The
reference arm runs on rank 0 only; the other ranks exit 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup(None)
        assert (w, r, local) == (world, rank, rank)
        slowest = bench.max_over_ranks(times[rank], dist, "cpu")
        assert slowest == max(times), (rank, slowest)
        # every rank reports the same job figure: all ranks' cells over the slowest time
        v = bench.job_mlups(4096 * 4096, 1000, world, slowest)
        assert v == pytest.approx(4096 * 4096 * 1000 * world / max(times) / 1e6)
        got = [None] * world
        dist.all_gather_object(got, v)
        assert len(set(got)) == 1
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    times = [0.75, 1.25]
    mp.spawn(_worker, args=(2, _free_port(), times), nprocs=2, join=True)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_mlups(100, 10, 1, 1e-3) == pytest.approx(1.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--side", "64", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 2
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_time_budget_bounds_the_sample():
    """The reference arm stops its timed oracle steps at the time budget and says
    how many of the requested steps it timed."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--side", "256", "--steps", "1000",
           "--warmup", "1", "--reference-budget-s", "0.2"]
    out = subprocess.run(cmd, cwd=ROOT, env=dict(os.environ, OMP_NUM_THREADS="2"), capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["steps"] == 1000 and 1 <= line["steps_timed"] < 1000
    assert line["cpu_baseline"]["sample"].startswith(f"{line['steps_timed']} of 1000 oracle steps")
    assert line["value"] > 0
