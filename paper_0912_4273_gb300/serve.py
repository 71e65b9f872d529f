"""Continuous-batching request loop for SimpleX2 solves on one GPU.

A request is a whole radiative-transfer solve: one grid, its sources, a bin
count, a time step and a number of steps.  The server

  * admits requests in arrival order while their device workspace (the HBM
    footprint reported by sx_workspace_bytes) fits in the memory budget, and
    keeps every admitted grid's state resident on the device;
  * advances admitted grids that share (bins, precision) together, a chunk
    of steps at a time, with one batched persistent launch per step
    (sx_batch_step); requests join and leave between chunks, so work of
    requests that arrived at different times overlaps on the device;
  * picks the grids of each chunk by least remaining work (steps left x
    vertices) until their vertices fill the device (``fill_vertices``): small
    grids share a launch, while a grid that fills the device alone is not
    slowed down by the others, which wait resident (shortest remaining work
    first keeps the median latency low); requests that have waited longer
    than ``max_wait_s`` since arrival go first, oldest first, so that large
    ones are not held back indefinitely;
  * loads newly admitted grids on their own stream while the others step;
  * reads a finished request's neutral fraction and photon budget, releases
    its workspace and records its latency (finish - arrival).

Failures are handled on the host: a request larger than the whole budget is
rejected, a load error fails that request only and returns its memory, a
chunk whose step fails (the worker "crashes") releases its requests and puts
them back at the head of the queue to start over, up to ``max_retries``
times, and a request can be cancelled while it waits or runs.

The device work goes through a backend object; ``GpuBackend`` is the real one
(the C ABI through ``simplex``); the tests drive the scheduling logic on the
CPU with a fake backend.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    problem: object            # inputs.Problem
    bins: np.ndarray           # nbins x 3 unit vectors
    steps: int
    dt: float
    seed: int = 0
    precision: int = 1         # simplex.SX_FP32_TRANSPORT
    arrival: float = 0.0       # seconds after the start of the run
    # filled in by the server
    status: str = "pending"    # pending | running | done | rejected | failed | cancelled
    error: str = ""
    y: Optional[np.ndarray] = None
    budget: Optional[dict] = None
    t_admit: float = float("nan")
    t_done: float = float("nan")
    retries: int = 0           # restarts after a failed chunk

    @property
    def nbins(self) -> int:
        return len(self.bins)

    @property
    def key(self):
        return (self.nbins, self.precision)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class GpuBackend:
    """Device side of the server: Solver contexts and Batch drivers."""

    def __init__(self, device: int = 0, max_grids: int = 256):
        import torch

        from . import simplex as S

        self.S = S
        self.torch = torch
        self.device = device
        self.max_grids = max_grids
        self.load_stream = torch.cuda.Stream(torch.device("cuda", device))
        self.streams = {}
        self.batches = {}

    def footprint(self, req: Request) -> int:
        s = self.S.Solver(req.bins, precision=req.precision, device=self.device,
                          stream=self.load_stream)
        try:
            return s.workspace_bytes(req.problem.n, req.problem.nnz)
        finally:
            s.close()

    def load(self, req: Request):
        s = self.S.Solver(req.bins, precision=req.precision, seed=req.seed, device=self.device,
                          stream=self.load_stream)
        s.load(req.problem)
        return s

    def step(self, key, solvers: List, dts: List[float], nsteps: int):
        if key not in self.batches:
            st = self.torch.cuda.Stream(self.torch.device("cuda", self.device))
            self.streams[key] = st
            self.batches[key] = self.S.Batch(self.max_grids, device=self.device, stream=st)
        self.batches[key].step(solvers, dts, nsteps)

    def finish(self, solver):
        y = solver.y
        b = solver.budget
        solver.close()
        return y, b

    def release(self, solver):
        solver.close()

    def close(self):
        for b in self.batches.values():
            b.close()
        self.batches.clear()


# Vertices that keep the step kernel busy: about four waves of its resident
# 32-vertex tiles (152 SMs x 6 CTAs) on a GB300.
DEFAULT_FILL_VERTICES = 1 << 17
# Waiting time after which a request goes ahead of shorter ones.
DEFAULT_MAX_WAIT_S = 1.0


class Server:
    """Continuous batching of SimpleX2 solves under an HBM budget."""

    def __init__(self, backend, hbm_budget: int, chunk_steps: int = 8, max_grids: int = 256,
                 clock: Callable[[], float] = time.perf_counter, first_fit: bool = True,
                 fill_vertices: Optional[int] = DEFAULT_FILL_VERTICES,
                 max_wait_s: Optional[float] = DEFAULT_MAX_WAIT_S, max_retries: int = 1):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.chunk = int(chunk_steps)
        self.max_grids = int(max_grids)
        self.clock = clock
        self.first_fit = first_fit
        self.fill = None if fill_vertices is None else int(fill_vertices)
        self.max_wait = None if max_wait_s is None else float(max_wait_s)
        self.max_retries = int(max_retries)
        self.pending: collections.deque = collections.deque()
        self.active: Dict[tuple, List[list]] = collections.defaultdict(list)  # key -> [[req, solver, done, bytes]]
        self.used = 0
        self.peak_used = 0
        self.finished: List[Request] = []
        self.t0 = None
        self._sizes: Dict[int, int] = {}

    # ----------------------------------------------------------------- API
    def submit(self, req: Request):
        self.pending.append(req)

    def cancel(self, rid: int) -> bool:
        for r in list(self.pending):
            if r.rid == rid:
                self.pending.remove(r)
                r.status = "cancelled"
                self.finished.append(r)
                return True
        for key, lst in self.active.items():
            for ent in lst:
                if ent[0].rid == rid:
                    lst.remove(ent)
                    self.backend.release(ent[1])
                    self.used -= ent[3]
                    ent[0].status = "cancelled"
                    self.finished.append(ent[0])
                    return True
        return False

    def now(self) -> float:
        return self.clock() - self.t0

    # ---------------------------------------------------------- scheduling
    def _size(self, req: Request) -> int:
        if req.rid not in self._sizes:
            self._sizes[req.rid] = int(self.backend.footprint(req))
        return self._sizes[req.rid]

    def _n_active(self) -> int:
        return sum(len(v) for v in self.active.values())

    def _admit(self):
        now = self.now()
        i = 0
        while i < len(self.pending):
            req = self.pending[i]
            if req.arrival > now:
                break
            need = self._size(req)
            if need > self.budget:
                del self.pending[i]
                req.status = "rejected"
                req.error = f"footprint {need} B exceeds the HBM budget {self.budget} B"
                req.t_done = now
                self.finished.append(req)
                continue
            if self.used + need <= self.budget and self._n_active() < self.max_grids:
                del self.pending[i]
                try:
                    solver = self.backend.load(req)
                except Exception as e:  # load failed: this request only
                    req.status = "failed"
                    req.error = str(e)
                    req.t_done = self.now()
                    self.finished.append(req)
                    continue
                self.used += need
                self.peak_used = max(self.peak_used, self.used)
                req.status = "running"
                req.t_admit = self.now()
                self.active[req.key].append([req, solver, 0, need])
                continue
            if not self.first_fit:
                break  # strict arrival order: later requests wait behind this one
            i += 1

    def _select(self, lst: List[list]) -> List[list]:
        """The grids of one key to advance in this chunk: requests past the
        maximum wait first (oldest first), then least remaining work, packed
        while their vertices stay within the fill target (at least one grid);
        every grid when there is no target."""
        if self.fill is None:
            return list(lst)
        now = self.now()

        def priority(ent):
            req = ent[0]
            if self.max_wait is not None and now - req.arrival > self.max_wait:
                return (0, req.arrival, req.rid)
            return (1, (req.steps - ent[2]) * req.problem.n, req.arrival, req.rid)

        order = sorted(lst, key=priority)
        picked, nv = [], 0
        for ent in order:
            if picked and nv + ent[0].problem.n > self.fill:
                continue
            picked.append(ent)
            nv += ent[0].problem.n
        return picked

    def _tick(self):
        for key in list(self.active.keys()):
            lst = self.active[key]
            if not lst:
                continue
            sel = self._select(lst)
            n = min(self.chunk, min(ent[0].steps - ent[2] for ent in sel))
            if n > 0:
                try:
                    self.backend.step(key, [ent[1] for ent in sel], [ent[0].dt for ent in sel], n)
                except Exception as e:  # the chunk failed: its requests start over
                    self._restart(lst, sel, str(e))
                    continue
                for ent in sel:
                    ent[2] += n
            done = [ent for ent in sel if ent[2] >= ent[0].steps]
            for ent in done:
                lst.remove(ent)
                req = ent[0]
                try:
                    req.y, req.budget = self.backend.finish(ent[1])
                    req.status = "done"
                except Exception as e:
                    req.status = "failed"
                    req.error = str(e)
                req.t_done = self.now()
                self.used -= ent[3]
                self.finished.append(req)

    def _restart(self, lst: List[list], sel: List[list], why: str):
        """Release the grids of a failed chunk; requeue their requests at the
        head of the queue (or fail those out of retries)."""
        requeue = []
        for ent in sel:
            lst.remove(ent)
            try:
                self.backend.release(ent[1])
            except Exception:
                pass
            self.used -= ent[3]
            req = ent[0]
            req.error = why
            if req.retries < self.max_retries:
                req.retries += 1
                req.status = "pending"
                requeue.append(req)
            else:
                req.status = "failed"
                req.t_done = self.now()
                self.finished.append(req)
        for req in sorted(requeue, key=lambda r: (r.arrival, r.rid), reverse=True):
            self.pending.appendleft(req)

    def run(self, requests=(), idle_sleep: float = 1e-4) -> List[Request]:
        """Serve ``requests`` (plus anything submitted before) to completion."""
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        self.t0 = self.clock()
        while self.pending or self._n_active():
            self._admit()
            if self._n_active():
                self._tick()
            elif self.pending:
                wait = self.pending[0].arrival - self.now()
                if wait > 0:
                    time.sleep(min(wait, 0.05) if idle_sleep else 0)
        return self.finished

    # ------------------------------------------------------------- metrics
    def stats(self) -> dict:
        done = [r for r in self.finished if r.status == "done"]
        lat = np.array([r.latency for r in done]) if done else np.zeros(0)
        span = max((r.t_done for r in done), default=0.0)
        return dict(
            solves=len(done), rejected=sum(r.status == "rejected" for r in self.finished),
            failed=sum(r.status == "failed" for r in self.finished),
            cancelled=sum(r.status == "cancelled" for r in self.finished),
            makespan_s=span, solves_per_s=len(done) / span if span > 0 else 0.0,
            p50_s=float(np.percentile(lat, 50)) if len(lat) else float("nan"),
            p99_s=float(np.percentile(lat, 99)) if len(lat) else float("nan"),
            peak_hbm_bytes=self.peak_used)


def serve_one_at_a_time(requests, device: int = 0, clock=time.perf_counter) -> dict:
    """The plain method: one grid per launch sequence, requests in arrival
    order, each stepped alone (sx_step) before the next is loaded."""
    import torch

    from . import simplex as S

    st = torch.cuda.Stream(torch.device("cuda", device))
    t0 = clock()
    out = []
    for r in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        s = S.Solver(r.bins, precision=r.precision, seed=r.seed, device=device, stream=st)
        s.load(r.problem)
        s.step(r.dt, r.steps)
        r.y, r.budget = s.y, s.budget
        s.close()
        r.t_done = clock() - t0
        r.status = "done"
        out.append(r)
    lat = np.array([r.latency for r in out])
    span = max(r.t_done for r in out)
    return dict(solves=len(out), makespan_s=span, solves_per_s=len(out) / span,
                p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)))
