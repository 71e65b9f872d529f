"""One grid split into shards, with a halo exchange after every step.

This is the paper's domain decomposition for distributed memory (Sect.
3.1-3.2): a vertex's step depends only on the photons its neighbours sent in
the previous step, so subdomains exchange their boundary once per step.

* ``partition`` splits the vertex ids (Morton-ordered by the generators, so
  a range is a compact region) into contiguous ranges with balanced edge
  counts: the shards' work.
* ``build_plans`` makes each shard's local grid -- its vertices plus, flagged
  SX_FLAG_GHOST, their neighbours on other shards, all in the whole grid's
  order, so that every row keeps its slot order -- and the exchange lists:
  for every ordered pair of shards (r, q), the masks and photon rows of r's
  vertices that q's gather reads, as r-local indices to pack and q-local
  indices to unpack, both in one canonical order (global sender, then global
  receiver).
* ``ShardedSolver`` steps the shards as contexts of this process (on one
  device or several) and moves the halos with device copies.
* ``exchange`` moves them between ``torch.distributed`` ranks, one shard per
  rank: NCCL with device buffers, or any backend (gloo) through host
  buffers.

The neutral fractions equal those of the whole grid bit for bit; the budget
terms, summed over the shards, to their rounding (the tiles' partial sums
group differently).  Direction-conserving transport only.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs as I

SX_FLAG_SINK = 1
SX_FLAG_GHOST = 2


def partition(row_ptr: np.ndarray, nparts: int) -> np.ndarray:
    """Boundaries b[0] = 0 < ... < b[nparts] = n of contiguous vertex ranges
    whose edge counts (the step kernel's work) are as equal as the ranges
    allow."""
    n = len(row_ptr) - 1
    if not 1 <= nparts <= n:
        raise ValueError("need 1 <= nparts <= n")
    work = row_ptr.astype(np.float64) + np.arange(n + 1)  # edges plus one per vertex
    targets = work[-1] * np.arange(1, nparts) / nparts
    cuts = np.searchsorted(work, targets)
    b = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    for k in range(1, nparts + 1):  # strictly increasing: no empty shard
        b[k] = max(b[k], b[k - 1] + 1)
    for k in range(nparts - 1, 0, -1):
        b[k] = min(b[k], b[k + 1] - 1)
    return b


@dataclasses.dataclass
class ShardPlan:
    rank: int
    nparts: int
    lo: int                   # owned global ids [lo, hi)
    hi: int
    glob: np.ndarray          # int64 [n_local]: global id of every local vertex (ascending)
    own0: int                 # local id of vertex lo (owned ids are own0 .. own0 + hi - lo - 1)
    problem: I.Problem        # the local grid (ghost flags set, owned sources only)
    send: dict                # peer -> (edge_idx int32, row_idx int32): r-local indices to pack
    recv: dict                # peer -> (edge_idx int32, row_idx int32): r-local indices to unpack

    @property
    def n_owned(self) -> int:
        return self.hi - self.lo


def _local_edge_index(row_ptr, col, a, b):
    """CSR index of each edge a -> b (local ids; every pair an edge)."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    keys = rows * n + col.astype(np.int64)          # ascending: rows, then sorted columns
    want = a.astype(np.int64) * n + b.astype(np.int64)
    idx = np.searchsorted(keys, want)
    if len(want) and not np.array_equal(keys[np.minimum(idx, len(keys) - 1)], want):
        raise ValueError("an exchanged pair is not an edge of the local grid")
    return idx


def build_plans(prob: I.Problem, nparts: int, bounds: np.ndarray | None = None) -> list[ShardPlan]:
    """Local grids and exchange lists of nparts shards of prob."""
    n = prob.n
    rp = np.asarray(prob.row_ptr, dtype=np.int64)
    col = np.asarray(prob.col, dtype=np.int64)
    b = partition(rp, nparts) if bounds is None else np.asarray(bounds, dtype=np.int64)
    owner = np.repeat(np.arange(nparts), np.diff(b))
    src_of_edge = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    locals_, plans = [], []
    for r in range(nparts):
        lo, hi = int(b[r]), int(b[r + 1])
        nbr = col[rp[lo]:rp[hi]]
        ghosts = np.unique(nbr[(nbr < lo) | (nbr >= hi)])
        glob = np.union1d(np.arange(lo, hi, dtype=np.int64), ghosts)
        is_local = np.zeros(n, dtype=bool)
        is_local[glob] = True
        loc_of = np.full(n, -1, dtype=np.int64)
        loc_of[glob] = np.arange(len(glob))
        # every local vertex's local neighbours, in the whole grid's order
        starts, ends = rp[glob], rp[glob + 1]
        cnt_all = ends - starts
        e_all = np.repeat(starts - np.concatenate([[0], np.cumsum(cnt_all)[:-1]]), cnt_all) + \
            np.arange(cnt_all.sum())
        nb_all = col[e_all]
        keep = is_local[nb_all]
        row_of = np.repeat(np.arange(len(glob)), cnt_all)[keep]
        lcol = loc_of[nb_all[keep]].astype(np.int32)
        lrp = np.zeros(len(glob) + 1, dtype=np.int64)
        np.add.at(lrp, row_of + 1, 1)
        lrp = np.cumsum(lrp)
        flags = np.asarray(prob.flags, dtype=np.uint8)[glob].copy()
        flags[(glob < lo) | (glob >= hi)] |= SX_FLAG_GHOST
        sv = np.asarray(prob.src_vertex, dtype=np.int64)
        mine = (sv >= lo) & (sv < hi)
        local = I.Problem(pos=np.ascontiguousarray(prob.pos[glob]), row_ptr=lrp, col=lcol,
                          nH=np.ascontiguousarray(prob.nH[glob]),
                          volume=np.ascontiguousarray(prob.volume[glob]), flags=flags,
                          src_vertex=loc_of[sv[mine]].astype(np.int32),
                          src_rate=np.asarray(prob.src_rate)[mine], box=prob.box,
                          meta=dict(prob.meta, shard=r, nparts=nparts))
        own0 = int(loc_of[lo])
        plans.append(ShardPlan(rank=r, nparts=nparts, lo=lo, hi=hi, glob=glob, own0=own0,
                               problem=local, send={}, recv={}))
        locals_.append(loc_of)
    # exchange lists: sender u owned by r, receiver v owned by q != r
    e_u, e_v = src_of_edge, col
    cross = owner[e_u] != owner[e_v]
    cu, cv = e_u[cross], e_v[cross]                    # ascending (u, v): CSR order
    ro, qo = owner[cu], owner[cv]
    for r in range(nparts):
        for q in range(nparts):
            if q == r:
                continue
            sel = (ro == r) & (qo == q)
            if not sel.any():
                continue
            u, v = cu[sel], cv[sel]
            rows = np.unique(u)                         # r's vertices that are ghosts on q
            pr, pq = plans[r], plans[q]
            lr, lq = locals_[r], locals_[q]
            # the mask of u -> v sits at v's in-edge from u: edge (v -> u)
            se = _local_edge_index(pr.problem.row_ptr, pr.problem.col, lr[v], lr[u])
            re = _local_edge_index(pq.problem.row_ptr, pq.problem.col, lq[v], lq[u])
            pr.send[q] = (se.astype(np.int32), lr[rows].astype(np.int32))
            pq.recv[r] = (re.astype(np.int32), lq[rows].astype(np.int32))
    return plans


def photon_unit(src_rate, dt: float) -> float:
    """The FP32 photon unit a whole grid with these sources takes at a first
    step of dt: the power of two just above the photons of one step."""
    tot = 0.0
    for r in np.asarray(src_rate, dtype=np.float64):
        tot += float(r) * dt
    if not tot > 0.0:
        return 1.0
    return math.ldexp(1.0, math.frexp(tot)[1])


def global_kappa(sums) -> float:
    """kappa of the whole grid from the shards' (num, den) (sx_kappa_sums)."""
    num = sum(s[0] for s in sums)
    den = sum(s[1] for s in sums)
    return num / den if den > 0 else 1.0


class ShardedSolver:
    """A grid split into ``nparts`` shards, each a context of this process
    (on ``devices[r % len(devices)]``), stepped together with a halo
    exchange after every step through device copies.  ``kappa`` <= 0: the
    whole grid's, from the shards' sums.  Other keywords go to each
    shard's :class:`~paper_0912_4273_gb300.simplex.Solver`."""

    def __init__(self, bins, prob: I.Problem, nparts: int, devices=(0,), kappa: float = 0.0,
                 bounds=None, **solver_kw):
        import torch

        from . import simplex as S

        self._torch, self._S = torch, S
        self.plans = build_plans(prob, nparts, bounds)
        self.n = prob.n
        self.src_rate = np.asarray(prob.src_rate, dtype=np.float64)
        self.started = False
        devs = [torch.device("cuda", d) for d in devices]
        self.devices = [devs[r % len(devs)] for r in range(nparts)]
        self.streams = [torch.cuda.Stream(d) for d in self.devices]
        if kappa <= 0.0:
            sums = []
            for p, d, st in zip(self.plans, self.devices, self.streams):
                t = S.Solver(bins, device=d.index, stream=st, **solver_kw).load(p.problem)
                sums.append(S.sx_kappa_sums(t.ctx))
                t.close()
            kappa = global_kappa(sums)
        self.kappa = kappa
        self.solvers = [S.Solver(bins, device=d.index, stream=st, kappa=kappa, **solver_kw).load(p.problem)
                        for p, d, st in zip(self.plans, self.devices, self.streams)]
        # per ordered pair: index arrays and a buffer on each side
        self.links = []
        for r, p in enumerate(self.plans):
            for q, (se, sr) in sorted(p.send.items()):
                re, rr = self.plans[q].recv[r]
                nbytes = S.sx_halo_bytes(self.solvers[r].ctx, len(se), len(sr))
                dr, dq = self.devices[r], self.devices[q]
                self.links.append(dict(
                    r=r, q=q, ne=len(se), nr=len(sr),
                    se=torch.from_numpy(se).to(dr), sr=torch.from_numpy(sr).to(dr),
                    re=torch.from_numpy(re).to(dq), rr=torch.from_numpy(rr).to(dq),
                    bs=torch.empty(nbytes, dtype=torch.uint8, device=dr),
                    bq=torch.empty(nbytes, dtype=torch.uint8, device=dq)))
        self.halo_bytes_per_step = sum(int(L["bs"].numel()) for L in self.links)

    def step(self, dt: float, nsteps: int = 1):
        S, torch = self._S, self._torch
        if not self.started:  # every shard stores photons in the whole grid's unit
            u = photon_unit(self.src_rate, dt)
            for s in self.solvers:
                S.sx_set_photon_unit(s.ctx, u)
            self.started = True
        for _ in range(nsteps):
            for s in self.solvers:
                s.step(dt, 1)
            for L in self.links:
                r, q = L["r"], L["q"]
                S.sx_halo_pack(self.solvers[r].ctx, L["ne"], L["se"].data_ptr(), L["nr"],
                               L["sr"].data_ptr(), L["bs"].data_ptr())
                ev = torch.cuda.Event()
                ev.record(self.streams[r])
                self.streams[q].wait_event(ev)
                with torch.cuda.stream(self.streams[q]):
                    L["bq"].copy_(L["bs"], non_blocking=True)
                S.sx_halo_unpack(self.solvers[q].ctx, L["ne"], L["re"].data_ptr(), L["nr"],
                                 L["rr"].data_ptr(), L["bq"].data_ptr())
                # the sender's next pack overwrites bs only after this copy
                ev2 = torch.cuda.Event()
                ev2.record(self.streams[q])
                self.streams[r].wait_event(ev2)

    def sync(self):
        for s in self.solvers:
            s.sync()

    @property
    def y(self) -> np.ndarray:
        out = np.empty(self.n)
        for p, s in zip(self.plans, self.solvers):
            out[p.lo:p.hi] = s.y[p.own0:p.own0 + p.n_owned]
        return out

    def photons(self) -> np.ndarray:
        out = np.empty(self.n)
        for p, s in zip(self.plans, self.solvers):
            out[p.lo:p.hi] = s.photons()[p.own0:p.own0 + p.n_owned]
        return out

    @property
    def budget(self) -> dict:
        tot = dict(emitted=0.0, absorbed=0.0, escaped=0.0, in_flight=0.0)
        for s in self.solvers:
            for k, v in s.budget.items():
                tot[k] += v
        return tot

    def close(self):
        for s in self.solvers:
            s.close()
        self.solvers = []


def exchange(plan: ShardPlan, pack, unpack, send_bufs: dict, recv_bufs: dict, group=None):
    """One halo exchange of this rank's shard with the other ranks of a
    ``torch.distributed`` group (rank r of the group holds shard r).

    pack(q, buf) fills send_bufs[q] with what shard q reads from this shard;
    unpack(q, buf) applies recv_bufs[q], received from shard q.  The buffers
    are tensors of the backend's kind (device tensors for NCCL, host
    tensors for gloo); the sends and receives are posted together and all
    complete before any unpack."""
    import torch.distributed as dist

    for q in sorted(plan.send):
        pack(q, send_bufs[q])
    ops = [dist.P2POp(dist.isend, send_bufs[q], q, group) for q in sorted(plan.send)]
    ops += [dist.P2POp(dist.irecv, recv_bufs[q], q, group) for q in sorted(plan.recv)]
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for q in sorted(plan.recv):
        unpack(q, recv_bufs[q])
