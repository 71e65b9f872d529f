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
  * loads newly admitted grids on a host thread and their own stream while
    the others step, and reads a finished request's neutral fraction and
    photon budget on another host thread once its last chunk has run, then
    releases its workspace and records its latency (results in hand -
    arrival); the main loop only queues chunks, at most ``max_inflight``
    ahead of the device, so the GPU is not left idle while the host loads or
    reads.

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
import concurrent.futures as cf
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

    def load_async(self, req: Request) -> cf.Future:
        """The load on the loader thread (sx_load_grid waits for its own
        stream only, so the batches keep running)."""
        return self._loader().submit(self.load, req)

    def step(self, key, solvers: List, dts: List[float], nsteps: int):
        """Queue a chunk; returns an event that completes with it."""
        if key not in self.batches:
            st = self.torch.cuda.Stream(self.torch.device("cuda", self.device))
            self.streams[key] = st
            self.batches[key] = self.S.Batch(self.max_grids, device=self.device, stream=st)
        self.batches[key].step(solvers, dts, nsteps)
        ev = self.torch.cuda.Event()
        ev.record(self.streams[key])
        return ev

    @staticmethod
    def done(event) -> bool:
        return event.query()

    @staticmethod
    def wait(event):
        event.synchronize()

    def finish(self, solver):
        y = solver.y
        b = solver.budget
        solver.close()
        return y, b

    def finish_async(self, solver) -> cf.Future:
        """The reads on the reader thread: they wait for the context's own
        stream, which waits for the chunks that stepped it, not for later
        chunks of other grids."""
        return self._reader().submit(self.finish, solver)

    def release(self, solver):
        solver.close()

    def _loader(self):
        if getattr(self, "_load_pool", None) is None:
            self._load_pool = cf.ThreadPoolExecutor(max_workers=1, thread_name_prefix="sx-load")
        return self._load_pool

    def _reader(self):
        if getattr(self, "_read_pool", None) is None:
            self._read_pool = cf.ThreadPoolExecutor(max_workers=1, thread_name_prefix="sx-read")
        return self._read_pool

    def close(self):
        for pool in (getattr(self, "_load_pool", None), getattr(self, "_read_pool", None)):
            if pool is not None:
                pool.shutdown(wait=True)
        self._load_pool = self._read_pool = None
        for b in self.batches.values():
            b.close()
        self.batches.clear()


def _done_future(fn, *args) -> cf.Future:
    """fn(*args) run now, as a completed future (backends without threads)."""
    f: cf.Future = cf.Future()
    try:
        f.set_result(fn(*args))
    except Exception as e:  # noqa: BLE001 -- handed to the caller through the future
        f.set_exception(e)
    return f


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
                 max_wait_s: Optional[float] = DEFAULT_MAX_WAIT_S, max_retries: int = 1,
                 max_inflight: int = 2):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.chunk = int(chunk_steps)
        self.max_grids = int(max_grids)
        self.clock = clock
        self.first_fit = first_fit
        self.fill = None if fill_vertices is None else int(fill_vertices)
        self.max_wait = None if max_wait_s is None else float(max_wait_s)
        self.max_retries = int(max_retries)
        self.max_inflight = max(1, int(max_inflight))
        self.pending: collections.deque = collections.deque()
        self.active: Dict[tuple, List[list]] = collections.defaultdict(list)  # key -> [[req, solver, done, bytes]]
        self.loading: List[list] = []    # [req, future of the solver, bytes]
        self.reading: List[list] = []    # [req, future of (y, budget), bytes]
        self.inflight: collections.deque = collections.deque()  # events of queued chunks
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
        for ent in list(self.loading):
            if ent[0].rid == rid:  # its load runs to the end, then the grid is released
                self.loading.remove(ent)
                try:
                    self.backend.release(ent[1].result())
                except Exception:
                    pass
                self.used -= ent[2]
                ent[0].status = "cancelled"
                self.finished.append(ent[0])
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

    def _n_resident(self) -> int:
        return self._n_active() + len(self.loading) + len(self.reading)

    def _load(self, req: Request) -> cf.Future:
        if hasattr(self.backend, "load_async"):
            return self.backend.load_async(req)
        return _done_future(self.backend.load, req)

    def _read(self, solver) -> cf.Future:
        if hasattr(self.backend, "finish_async"):
            return self.backend.finish_async(solver)
        return _done_future(self.backend.finish, solver)

    def _collect_loads(self):
        keep = []
        for req, fut, need in self.loading:
            if not fut.done():
                keep.append([req, fut, need])
                continue
            try:
                solver = fut.result()
            except Exception as e:  # load failed: this request only
                self.used -= need
                req.status = "failed"
                req.error = str(e)
                req.t_done = self.now()
                self.finished.append(req)
                continue
            req.status = "running"
            self.active[req.key].append([req, solver, 0, need])
        self.loading = keep

    def _collect_reads(self):
        keep = []
        for req, fut, need in self.reading:
            if not fut.done():
                keep.append([req, fut, need])
                continue
            try:
                req.y, req.budget = fut.result()
                req.status = "done"
            except Exception as e:
                req.status = "failed"
                req.error = str(e)
            req.t_done = self.now()
            self.used -= need
            self.finished.append(req)
        self.reading = keep

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
            if self.used + need <= self.budget and self._n_resident() < self.max_grids:
                del self.pending[i]
                self.used += need
                self.peak_used = max(self.peak_used, self.used)
                req.status = "loading"
                req.t_admit = self.now()
                self.loading.append([req, self._load(req), need])
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

    def _throttle(self):
        """At most max_inflight chunks queued ahead of the device."""
        while self.inflight and (len(self.inflight) >= self.max_inflight
                                 or getattr(self.backend, "done", lambda e: True)(self.inflight[0])):
            ev = self.inflight.popleft()
            if hasattr(self.backend, "wait"):
                self.backend.wait(ev)

    def _tick(self):
        for key in list(self.active.keys()):
            lst = self.active[key]
            if not lst:
                continue
            sel = self._select(lst)
            n = min(self.chunk, min(ent[0].steps - ent[2] for ent in sel))
            if n > 0:
                self._throttle()
                try:
                    ev = self.backend.step(key, [ent[1] for ent in sel], [ent[0].dt for ent in sel], n)
                except Exception as e:  # the chunk failed: its requests start over
                    self._restart(lst, sel, str(e))
                    continue
                if ev is not None:
                    self.inflight.append(ev)
                for ent in sel:
                    ent[2] += n
            done = [ent for ent in sel if ent[2] >= ent[0].steps]
            for ent in done:  # its results are read on the reader thread
                lst.remove(ent)
                ent[0].status = "reading"
                self.reading.append([ent[0], self._read(ent[1]), ent[3]])

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
        while self.pending or self._n_resident():
            self._admit()
            self._collect_loads()
            if self._n_active():
                self._tick()
            self._collect_reads()
            if not self._n_active():
                if self.loading or self.reading:  # wait for the host threads
                    futs = [f for _, f, _ in self.loading + self.reading]
                    cf.wait(futs, timeout=0.05, return_when=cf.FIRST_COMPLETED)
                elif self.pending:
                    wait = self.pending[0].arrival - self.now()
                    if wait > 0:
                        time.sleep(min(wait, 0.05) if idle_sleep else 0)
        while self.inflight:
            ev = self.inflight.popleft()
            if hasattr(self.backend, "wait"):
                self.backend.wait(ev)
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
