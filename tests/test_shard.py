"""Shards of one grid (host side, no GPU): the partition, the local grids and
the halo-exchange lists, in process and between two gloo ranks.

The step kernels are emulated by what they leave behind: every owned vertex
u writes, for each out-edge u -> v, a mask coding (u, v) at v's in-edge from
u and a photon row coding u.  After one exchange every owned vertex must see,
on every in-edge, its sender's mask and row -- whether the sender is on the
same shard or not."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_0912_4273_gb300 import inputs as I
from paper_0912_4273_gb300 import shard as SH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MW, NBP = 4, 8   # mask words per edge and photon-row width of the emulation


def _mask(u, v):
    c = (np.asarray(u, np.uint64) * np.uint64(1000003) + np.asarray(v, np.uint64)) & np.uint64(0xFFFFFFFF)
    return np.stack([c + np.uint64(k) for k in range(MW)], axis=-1).astype(np.uint32)


def _row(u):
    return np.asarray(u, np.float64)[..., None] + np.arange(NBP) / 16.0


def owner_view(plan):
    """The buffers after a step: masks and rows of the shard's own vertices."""
    p = plan.problem
    rp, col = np.asarray(p.row_ptr), np.asarray(p.col)
    n_loc = len(plan.glob)
    M = np.zeros((len(col), MW), np.uint32)
    P = np.zeros((n_loc, NBP))
    own = np.arange(plan.own0, plan.own0 + plan.n_owned)
    a = np.repeat(np.arange(n_loc), np.diff(rp))
    sel = (a >= plan.own0) & (a < plan.own0 + plan.n_owned)
    u, v = a[sel], col[sel]
    tw = SH._local_edge_index(rp, col, v, u)  # the mask of u -> v sits at v's in-edge (v -> u)
    M[tw] = _mask(plan.glob[u], plan.glob[v])
    P[own] = _row(plan.glob[own])
    return M, P


def pack(plan, M, P, q):
    se, sr = plan.send[q]
    return M[se].copy(), P[sr].copy()


def unpack(plan, M, P, r, data):
    re, rr = plan.recv[r]
    M[re], P[rr] = data


def check_receivers(plan, M, P):
    p = plan.problem
    rp, col = np.asarray(p.row_ptr), np.asarray(p.col)
    a = np.repeat(np.arange(len(plan.glob)), np.diff(rp))
    sel = (a >= plan.own0) & (a < plan.own0 + plan.n_owned)
    v, u = a[sel], col[sel]                   # owned receiver v, its senders u
    e = np.nonzero(sel)[0]                    # v's in-edge from u
    assert np.array_equal(M[e], _mask(plan.glob[u], plan.glob[v]))
    assert np.array_equal(P[u], _row(plan.glob[u]))


@pytest.fixture(scope="module")
def grid():
    return I.stromgren_problem(3000, seed=4)


def test_partition_balances_edges(grid):
    b = SH.partition(grid.row_ptr, 4)
    assert b[0] == 0 and b[-1] == grid.n and np.all(np.diff(b) > 0)
    w = np.diff(grid.row_ptr[b] + b)
    assert w.max() / w.mean() < 1.02


@pytest.mark.parametrize("nparts", [2, 3, 5])
def test_local_grids_keep_the_rows_of_the_whole_grid(grid, nparts):
    plans = SH.build_plans(grid, nparts)
    assert sum(p.n_owned for p in plans) == grid.n
    for p in plans:
        lp = p.problem
        rp, col = np.asarray(lp.row_ptr), np.asarray(lp.col)
        assert np.all(np.diff(p.glob) > 0)                  # the whole grid's order
        own = np.arange(p.own0, p.own0 + p.n_owned)
        assert np.array_equal(p.glob[own], np.arange(p.lo, p.hi))
        ghost = (lp.flags & SH.SX_FLAG_GHOST) != 0
        assert not ghost[own].any() and ghost.sum() == len(p.glob) - p.n_owned
        for i in range(len(p.glob)):
            row = p.glob[col[rp[i]:rp[i + 1]]]
            g = p.glob[i]
            full = grid.col[grid.row_ptr[g]:grid.row_ptr[g + 1]]
            if not ghost[i]:
                assert np.array_equal(row, full)            # every neighbour, in slot order
            else:
                assert np.array_equal(row, full[np.isin(full, p.glob)])
        # symmetric local CSR
        a = np.repeat(np.arange(len(p.glob)), np.diff(rp))
        SH._local_edge_index(rp, col, col, a)
        # sources on their owner only
        assert np.all((lp.src_vertex >= p.own0) & (lp.src_vertex < p.own0 + p.n_owned))
    assert sum(len(p.problem.src_vertex) for p in plans) == len(grid.src_vertex)


@pytest.mark.parametrize("nparts", [2, 3, 4])
def test_exchange_delivers_every_remote_sender(grid, nparts):
    plans = SH.build_plans(grid, nparts)
    bufs = [owner_view(p) for p in plans]
    for r, p in enumerate(plans):
        for q in p.send:
            unpack(plans[q], *bufs[q], r, pack(p, *bufs[r], q))
    for p, (M, P) in zip(plans, bufs):
        check_receivers(p, M, P)


def test_exchange_lists_agree_in_length(grid):
    plans = SH.build_plans(grid, 3)
    for r, p in enumerate(plans):
        for q, (se, sr) in p.send.items():
            re, rr = plans[q].recv[r]
            assert len(se) == len(re) and len(sr) == len(rr)


def test_global_kappa_is_the_ratio_of_summed_sums():
    assert SH.global_kappa([(1.0, 2.0), (3.0, 4.0)]) == pytest.approx(4.0 / 6.0)


WORKER = r'''
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
import numpy as np
import torch
import torch.distributed as dist
from paper_0912_4273_gb300 import inputs as I
from paper_0912_4273_gb300 import shard as SH
import test_shard as T
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
grid = I.stromgren_problem(3000, seed=4)
plan = SH.build_plans(grid, world)[rank]
M, P = T.owner_view(plan)

def nbytes(ne, nr):
    return ne * T.MW * 4 + nr * T.NBP * 8

def pack(q, buf):
    m, p = T.pack(plan, M, P, q)
    buf.copy_(torch.frombuffer(bytearray(m.tobytes() + p.tobytes()), dtype=torch.uint8))

def unpack(q, buf):
    re, rr = plan.recv[q]
    b = buf.numpy().tobytes()
    m = np.frombuffer(b[:len(re) * T.MW * 4], np.uint32).reshape(len(re), T.MW)
    p = np.frombuffer(b[len(re) * T.MW * 4:], np.float64).reshape(len(rr), T.NBP)
    T.unpack(plan, M, P, q, (m, p))

send = {q: torch.empty(nbytes(len(se), len(sr)), dtype=torch.uint8) for q, (se, sr) in plan.send.items()}
recv = {q: torch.empty(nbytes(len(re), len(rr)), dtype=torch.uint8) for q, (re, rr) in plan.recv.items()}
SH.exchange(plan, pack, unpack, send, recv)
T.check_receivers(plan, M, P)
print(json.dumps({"rank": rank, "ghost_rows": int(sum(len(v[1]) for v in plan.recv.values()))}))
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_between_gloo_ranks(world):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    assert sorted(r["rank"] for r in res) == list(range(world))
    assert all(r["ghost_rows"] > 0 for r in res)
