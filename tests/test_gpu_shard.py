"""Shards of one grid on the GPU (Sect. 3.1-3.2: one halo exchange per step).

The grid is split into 2 or 3 shards, each a context with its ghosts; after
every step each shard's halo goes to the others (sx_halo_pack -> copy ->
sx_halo_unpack).  Against the whole grid run as one context with the same
kappa: the neutral fractions and the photons in flight towards every vertex
are equal bit for bit (every vertex gathers its packets in the same order),
the budget terms summed over the shards to 1e-12 of the emitted photons
(the tiles group the sums differently).  kappa from the shards' sums matches
the whole grid's, and the sharded FP64 solve matches the oracle at 1e-9.
Also run as two processes on one GPU, exchanging through host memory over
gloo (blocking host transfers between the steps; no kernel waits on
another)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import shard as SH  # noqa: E402
from paper_0912_4273_gb300 import simplex as S  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DT = 2.5 * I.MYR_S


def _budget_err(b, rb):
    return max(abs(b[k] - rb[k]) for k in rb) / rb["emitted"]


@pytest.fixture(scope="module")
def grid():
    return I.stromgren_problem(6000, seed=9)


@pytest.mark.parametrize("nparts", [2, 3])
@pytest.mark.parametrize("precision", [S.SX_FP64, S.SX_FP32_TRANSPORT])
def test_shards_equal_the_whole_grid(grid, nparts, precision):
    bins = I.fibonacci_bins(42)
    one = S.Solver(bins, precision=precision, seed=9).load(grid)
    kappa = one.info["kappa"]
    sh = SH.ShardedSolver(bins, grid, nparts, kappa=kappa, precision=precision, seed=9)
    assert sh.halo_bytes_per_step > 0
    for steps in (1, 15, 24):
        one.step(DT, steps)
        sh.step(DT, steps)
        assert np.array_equal(sh.y, one.y)
        assert np.array_equal(sh.photons(), one.photons())
        assert _budget_err(sh.budget, one.budget) <= 1e-12
    for s in sh.solvers:
        assert s.info["index_errors"] == 0
    sh.close()
    one.close()


def test_kappa_from_the_shards_sums(grid):
    bins = I.fibonacci_bins(84)
    one = S.Solver(bins, precision=S.SX_FP32_TRANSPORT).load(grid)
    sh = SH.ShardedSolver(bins, grid, 3)
    assert sh.kappa == pytest.approx(one.info["kappa"], rel=1e-12)
    sh.close()
    one.close()


def test_sharded_clumpy_medium_matches_the_oracle():
    prob = I.clumpy_problem(6000, seed=3)  # 16 sources, spread over the shards
    bins = I.fibonacci_bins(42)
    ref = O.OracleSim(prob, O.Params(nbins=42, seed=3), bins)
    sh = SH.ShardedSolver(bins, prob, 3, kappa=ref.kappa, precision=S.SX_FP64, seed=3)
    assert sum(len(p.problem.src_vertex) for p in sh.plans) == 16
    for steps in (10, 20):
        ref.step(0.5 * I.MYR_S, steps)
        sh.step(0.5 * I.MYR_S, steps)
        assert np.abs(sh.y - ref.y).max() <= 1e-9
        assert _budget_err(sh.budget, ref.budget) <= 1e-9
    sh.close()


def test_halo_calls_check_their_arguments(grid):
    s = S.Solver(I.fibonacci_bins(42)).load(grid)
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SimplexError) as e:  # no step yet: nothing to exchange
        S.sx_halo_pack(s.ctx, 1, d.data_ptr(), 0, 0, d.data_ptr())
    assert e.value.code == S.SX_ESTATE
    s.step(DT, 1)
    with pytest.raises(S.SimplexError):
        S.sx_halo_pack(s.ctx, -1, d.data_ptr(), 0, 0, d.data_ptr())
    # indices out of range are skipped and counted, not used
    bad = torch.tensor([2 ** 30, -5], dtype=torch.int32, device="cuda")
    buf = torch.zeros(S.sx_halo_bytes(s.ctx, 2, 0), dtype=torch.uint8, device="cuda")
    S.sx_halo_unpack(s.ctx, 2, bad.data_ptr(), 0, 0, buf.data_ptr())
    s.sync()
    assert s.info["index_errors"] == 2
    s.close()
    b = S.Solver(I.fibonacci_bins(42), transport=S.SX_TRANSPORT_BALLISTIC).load(grid)
    b.step(DT, 1)
    with pytest.raises(S.SimplexError):
        S.sx_halo_pack(b.ctx, 0, 0, 0, 0, 0)
    b.close()


WORKER = r'''
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch
import torch.distributed as dist
from paper_0912_4273_gb300 import inputs as I
from paper_0912_4273_gb300 import shard as SH
from paper_0912_4273_gb300 import simplex as S
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
grid = I.stromgren_problem(6000, seed=9)
plan = SH.build_plans(grid, world)[rank]
bins = I.fibonacci_bins(42)
kappa = float(os.environ["KAPPA"])
st = torch.cuda.Stream()
s = S.Solver(bins, precision=S.SX_FP64, seed=9, kappa=kappa, stream=st).load(plan.problem)
dev = {}
for q, (se, sr) in plan.send.items():
    dev[("s", q)] = (torch.from_numpy(se).cuda(), torch.from_numpy(sr).cuda(),
                     torch.empty(S.sx_halo_bytes(s.ctx, len(se), len(sr)), dtype=torch.uint8, device="cuda"))
for q, (re, rr) in plan.recv.items():
    dev[("r", q)] = (torch.from_numpy(re).cuda(), torch.from_numpy(rr).cuda(),
                     torch.empty(S.sx_halo_bytes(s.ctx, len(re), len(rr)), dtype=torch.uint8, device="cuda"))
send = {q: torch.empty(dev[("s", q)][2].numel(), dtype=torch.uint8).pin_memory() for q in plan.send}
recv = {q: torch.empty(dev[("r", q)][2].numel(), dtype=torch.uint8).pin_memory() for q in plan.recv}

def pack(q, host):
    e, r, b = dev[("s", q)]
    S.sx_halo_pack(s.ctx, e.numel(), e.data_ptr(), r.numel(), r.data_ptr(), b.data_ptr())
    with torch.cuda.stream(st):
        host.copy_(b, non_blocking=True)
    st.synchronize()

def unpack(q, host):
    e, r, b = dev[("r", q)]
    with torch.cuda.stream(st):
        b.copy_(host, non_blocking=True)
    S.sx_halo_unpack(s.ctx, e.numel(), e.data_ptr(), r.numel(), r.data_ptr(), b.data_ptr())
    st.synchronize()  # the host buffer is reused by the next exchange

S.sx_set_photon_unit(s.ctx, SH.photon_unit(grid.src_rate, 2.5 * I.MYR_S))
for _ in range(int(os.environ["STEPS"])):
    s.step(2.5 * I.MYR_S, 1)
    SH.exchange(plan, pack, unpack, send, recv)
y = s.y[plan.own0:plan.own0 + plan.n_owned]
b = s.budget
np.save(os.path.join(os.environ["OUT"], f"y{rank}.npy"), y)
print(json.dumps({"rank": rank, "lo": plan.lo, "hi": plan.hi, "budget": b}))
s.close()
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_processes_exchange_over_gloo(grid, tmp_path):
    bins = I.fibonacci_bins(42)
    one = S.Solver(bins, precision=S.SX_FP64, seed=9).load(grid)
    kappa = one.info["kappa"]
    steps = 30
    one.step(DT, steps)
    y_one, b_one = one.y, one.budget
    one.close()
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), ROOT=ROOT, KAPPA=repr(kappa), STEPS=str(steps), OUT=str(tmp_path))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-3000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda d: d["rank"])
    y = np.concatenate([np.load(tmp_path / f"y{r['rank']}.npy") for r in res])
    assert np.array_equal(y, y_one)
    tot = {k: sum(r["budget"][k] for r in res) for k in b_one}
    assert _budget_err(tot, b_one) <= 1e-12
