"""bench.py's multi-rank path on CPU (gloo, world size 2).

Every rank runs its own replica; the only collectives are a barrier and the
max over the ranks' timings, and the whole-job value is the units of all
ranks over the slowest rank's time.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import bench
rank, world, local = bench.dist_env()
bench.dist_init(world, "gloo")
bench.barrier(world)
mine = 10.0 + 5.0 * rank
mx = bench.reduce_max(mine, world)
val = bench.aggregate(1000, world, mx)
bench.barrier(world)
print(json.dumps({"rank": rank, "max": mx, "value": val}))
import torch.distributed as dist
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_take_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["max"] == 15.0
        assert r["value"] == pytest.approx(2 * 1000 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    wl = bench.WORKLOADS["c0"]

    class A:
        steps, warmup = 1, 1

    bench.run_reference(A, wl, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_single_rank_helpers_are_identity():
    import bench

    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(10, 1, 1000.0) == 10.0


def test_grid_pools_built_on_worker_processes_match_direct_builds():
    """The served and batched benches build their grid pools on spawned
    worker processes (largest first); every grid must come back under its
    own key, equal to a build in this process."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from paper_0912_4273_gb300 import inputs as I

    jobs = [("stromgren_problem", 1500, 11), ("clumpy_problem", 3000, 12), ("stromgren_problem", 2500, 13)]
    built = bench._build_problems(jobs)
    for (recipe, n, seed), p in zip(jobs, built):
        q = getattr(I, recipe)(n, seed=seed)
        assert p.n == q.n and np.array_equal(p.col, q.col) and np.array_equal(p.pos, q.pos)
