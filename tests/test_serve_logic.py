"""Host-side logic of the serving loop, on the CPU with a fake backend:
admission by HBM footprint, continuous batching by (bins, precision), the
choice of grids per chunk (least remaining work within a fill target),
rejection, load failures, cancellation."""
import numpy as np
import pytest

from paper_0912_4273_gb300 import serve as SV


class FakeProblem:
    def __init__(self, n):
        self.n = n
        self.nnz = 16 * n


class FakeBackend:
    """Steps are counted, not computed; footprint = 100 B per vertex."""

    def __init__(self, fail_rids=()):
        self.steps = []        # (key, [rids], nsteps)
        self.loaded = []
        self.released = []
        self.fail = set(fail_rids)

    def footprint(self, req):
        return 100 * req.problem.n

    def load(self, req):
        if req.rid in self.fail:
            raise RuntimeError("simulated out of memory")
        self.loaded.append(req.rid)
        return {"rid": req.rid, "steps": 0}

    def step(self, key, solvers, dts, n):
        self.steps.append((key, [s["rid"] for s in solvers], n))
        for s in solvers:
            s["steps"] += n

    def finish(self, s):
        self.released.append(s["rid"])
        return np.full(3, float(s["steps"])), {"emitted": 1.0}

    def release(self, s):
        self.released.append(s["rid"])


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def req(rid, n, steps, nbins=42, arrival=0.0):
    return SV.Request(rid=rid, problem=FakeProblem(n), bins=np.zeros((nbins, 3)), steps=steps,
                      dt=1.0, arrival=arrival)


def test_admission_respects_the_hbm_budget_and_batches_by_key():
    be = FakeBackend()
    srv = SV.Server(be, hbm_budget=100 * 3000, chunk_steps=8, clock=Clock())
    rs = [req(0, 1000, 20), req(1, 1500, 12), req(2, 1000, 30, nbins=84), req(3, 400, 5)]
    out = srv.run(rs)
    assert all(r.status == "done" for r in out)
    assert srv.peak_used <= 100 * 3000
    # every grid got exactly its number of steps
    for r in out:
        assert r.y[0] == r.steps
    # request 2 (84 bins) never shares a launch with 42-bin grids
    for key, rids, n in be.steps:
        assert all(key == ((84, 1) if rid == 2 else (42, 1)) for rid in rids)
    # first fit: request 3 (small) passes request 2, which waits until memory frees
    by = {r.rid: r for r in out}
    assert by[3].t_admit < by[2].t_admit
    assert by[2].t_admit > min(by[0].t_done, by[1].t_done, by[3].t_done)
    assert srv.used == 0
    st = srv.stats()
    assert st["solves"] == 4 and st["p99_s"] >= st["p50_s"] > 0


def test_continuous_batching_joins_running_requests():
    be = FakeBackend()
    srv = SV.Server(be, hbm_budget=10**9, chunk_steps=4, clock=Clock())
    srv.run([req(0, 100, 40), req(1, 100, 8, arrival=0.005)])
    together = [rids for _, rids, _ in be.steps if len(rids) == 2]
    assert together, "the later request must join the running batch"


def test_least_remaining_work_first_within_the_fill_target():
    be = FakeBackend()
    srv = SV.Server(be, hbm_budget=10**9, chunk_steps=4, clock=Clock(), fill_vertices=1000)
    out = srv.run([req(0, 1000, 40), req(1, 100, 8, arrival=0.005), req(2, 300, 12, arrival=0.005)])
    by = {r.rid: r for r in out}
    assert all(r.status == "done" and r.y[0] == r.steps for r in out)
    # the small requests pass the large one, which fills the device alone
    assert by[1].t_done < by[0].t_done and by[2].t_done < by[0].t_done
    for _, rids, _ in be.steps:
        assert 0 not in rids or rids == [0]
    # the two small ones share launches (400 vertices within the target),
    # the one with less remaining work first
    shared = [rids for _, rids, _ in be.steps if len(rids) == 2]
    assert shared and all(rids == [1, 2] for rids in shared)
    # without a target every resident grid advances in every chunk
    be = FakeBackend()
    srv = SV.Server(be, hbm_budget=10**9, chunk_steps=4, clock=Clock(), fill_vertices=None)
    srv.run([req(0, 1000, 40), req(1, 100, 8, arrival=0.005)])
    assert any(sorted(rids) == [0, 1] for _, rids, _ in be.steps)


def test_a_request_past_the_maximum_wait_goes_first():
    # request 1 has less remaining work, but once both have waited longer
    # than max_wait the older one (request 0, lower id at equal arrival) leads
    def run(max_wait):
        be = FakeBackend()
        srv = SV.Server(be, hbm_budget=10**9, chunk_steps=4, clock=Clock(), fill_vertices=1000,
                        max_wait_s=max_wait)
        out = srv.run([req(0, 1000, 40), req(1, 900, 8)])
        assert all(r.status == "done" and r.y[0] == r.steps for r in out)
        assert all(len(rids) == 1 for _, rids, _ in be.steps)  # 1900 > 1000: never together
        return {r.rid: r.t_done for r in out}

    t = run(None)
    assert t[1] < t[0]
    t = run(0.002)
    assert t[0] < t[1]


class CrashingBackend(FakeBackend):
    """The step of chunk number `crash_at` fails (a worker crash)."""

    def __init__(self, crash_at, times=1):
        super().__init__()
        self.calls = 0
        self.crash_at = crash_at
        self.times = times

    def step(self, key, solvers, dts, n):
        self.calls += 1
        if self.crash_at <= self.calls < self.crash_at + self.times:
            raise RuntimeError("worker crashed")
        super().step(key, solvers, dts, n)


def test_a_crashed_chunk_restarts_its_requests():
    be = CrashingBackend(crash_at=2)
    srv = SV.Server(be, hbm_budget=10**9, chunk_steps=4, clock=Clock())
    out = srv.run([req(0, 100, 12), req(1, 200, 9)])
    by = {r.rid: r for r in out}
    assert all(r.status == "done" for r in out)
    # restarted from a fresh load: exactly its steps, once more loaded
    assert all(r.y[0] == r.steps for r in out)
    assert all(r.retries == 1 and "crashed" in r.error for r in out)
    assert sorted(be.loaded) == [0, 0, 1, 1]
    assert srv.used == 0
    # out of retries: failed, memory returned
    be = CrashingBackend(crash_at=1, times=10)
    srv = SV.Server(be, hbm_budget=10**9, chunk_steps=4, clock=Clock(), max_retries=2)
    out = srv.run([req(0, 100, 12)])
    assert out[0].status == "failed" and out[0].retries == 2 and srv.used == 0
    assert be.released.count(0) == 3


def test_rejection_failure_and_cancellation():
    be = FakeBackend(fail_rids={1})
    srv = SV.Server(be, hbm_budget=100 * 1000, clock=Clock())
    srv.submit(req(5, 10, 100, arrival=1e9))  # far in the future, cancelled before it arrives
    assert srv.cancel(5)
    out = srv.run([req(0, 5000, 10), req(1, 100, 10), req(2, 100, 10)])
    st = {r.rid: r.status for r in out}
    assert st == {5: "cancelled", 0: "rejected", 1: "failed", 2: "done"}
    assert srv.used == 0
    assert "exceeds" in next(r for r in out if r.rid == 0).error


def test_cancel_a_running_request_releases_its_memory():
    be = FakeBackend()
    srv = SV.Server(be, hbm_budget=10**9, clock=Clock())
    srv.t0 = 0.0
    srv.submit(req(0, 100, 1000))
    srv._admit()
    assert srv.used == 100 * 100
    assert srv.cancel(0)
    assert srv.used == 0 and be.released == [0]


class FakeEvent:
    def __init__(self, log):
        self.log = log
        self.waited = False

    def query(self):
        return self.waited


class AsyncFakeBackend(FakeBackend):
    """Loads and reads on host threads (with a delay), chunks as events that
    complete when waited for; counts the chunks queued ahead of the device."""

    def __init__(self, fail_rids=(), delay=0.002):
        super().__init__(fail_rids)
        import concurrent.futures as cf
        self.pool = cf.ThreadPoolExecutor(max_workers=2)
        self.delay = delay
        self.queued = []
        self.max_queued = 0

    def load_async(self, req):
        import time

        def work():
            time.sleep(self.delay)
            return self.load(req)
        return self.pool.submit(work)

    def finish_async(self, s):
        return self.pool.submit(self.finish, s)

    def step(self, key, solvers, dts, n):
        super().step(key, solvers, dts, n)
        ev = FakeEvent(self)
        self.queued.append(ev)
        self.max_queued = max(self.max_queued, sum(not e.waited for e in self.queued))
        return ev

    @staticmethod
    def done(ev):
        return ev.query()

    @staticmethod
    def wait(ev):
        ev.waited = True


def test_async_loads_and_reads_complete_every_request():
    be = AsyncFakeBackend(fail_rids=(3,))
    srv = SV.Server(be, hbm_budget=100 * 5000, chunk_steps=4, max_inflight=2,
                    clock=__import__("time").perf_counter)
    rs = [req(i, 500 + 300 * i, 10 + 3 * i, nbins=42 if i % 2 else 84, arrival=0.001 * i)
          for i in range(8)]
    out = srv.run(rs)
    by = {r.rid: r for r in out}
    assert by[3].status == "failed" and "simulated" in by[3].error
    for r in out:
        if r.rid != 3:
            assert r.status == "done" and r.y[0] == r.steps
    assert srv.used == 0 and not srv.loading and not srv.reading
    assert srv.peak_used <= srv.budget
    assert be.max_queued <= 2  # never more than max_inflight chunks ahead of the device
    assert sorted(be.released) == sorted(r.rid for r in out if r.status == "done")


def test_cancel_while_loading_releases_the_grid():
    be = AsyncFakeBackend(delay=0.05)
    srv = SV.Server(be, hbm_budget=100 * 5000, clock=__import__("time").perf_counter)
    srv.t0 = srv.clock()
    srv.submit(req(7, 1000, 5))
    srv._admit()
    assert srv.loading and srv.used == 100 * 1000
    assert srv.cancel(7)
    assert srv.used == 0 and not srv.loading and be.released == [7]
