"""CPU checks of bench.py's multi-process (replica) path: world-size-2 gloo
ranks agree on the max-over-ranks time, the whole-job value counts every
rank's work, and under torchrun only rank 0 runs and prints the CPU reference
arm.  (Every rank solves its own system: the factorisation has no independent
units to shard, so the N > 1 path is replicas only.)"""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (1 + r) seconds for the mixed path, 10 - r for FP64
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.0], world)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, 29571
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 0.0]


def test_replica_value_counts_all_ranks():
    F = bench.nominal_flops(16384, 64)
    one = bench.replica_value(1, F, 5, 0.25)
    assert bench.replica_value(4, F, 5, 0.25) == pytest.approx(4 * one)
    assert one == pytest.approx(F * 5 / 0.25 / 1e12)


def _run_bench(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_only_rank0_prints():
    r = _run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--impl", "reference",
                   "--workload", "c1", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    r = _run_bench({"RANK": "0", "WORLD_SIZE": "1"}, "--impl", "reference", "--workload", "c1",
                   "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "TFLOP/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
