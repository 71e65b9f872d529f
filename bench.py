#!/usr/bin/env python
"""Benchmark of the SimpleX2 DCT sweep on GB300.

Metric: DCT vertex-direction updates per second (interior vertices x bins x
steps / time) on the Test-1 Stromgren workload at 2^20 interior vertices and
84 bins: photons and transport in FP32 (compensated per-bin gathers), the
neutral fraction and the recombination subcycling in FP64, the budget's
global reduction in FP64.  One step is one pass of the whole hot path:
rotation and bin remap, gather, sources, chemistry, association and routing,
budget.  The grid is first advanced, untimed, to a fixed mid-run state
(--state-step, default step 300 of the 1000-step run), so that the timed
steps cost what the run's steps cost on average whatever --steps is.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica (its own grid and
seed): the path has no data exchange between GPUs, so scaling is weak and
the only collectives are a barrier and a max over the ranks' timings.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DCT vertex-direction updates/s"
UNIT = "updates/s"

WORKLOADS = {
    # 2^20 interior vertices of the Test-1 grid (Sect. 5.1), 84 bins, 1000 steps over 500 Myr
    "c1": dict(n=1 << 20, nbins=84, precision="fp32", dt_myr=0.5, seed=0, run_steps=1000,
               name="Test-1 Stromgren problem: 2^20 interior Poisson-Delaunay vertices in the "
                    "13.2 kpc mirror box of the 6.6 kpc corner-source cube (source at the centre) "
                    "+ sink shell, 84 direction bins, 1000 steps of 0.5 Myr"),
    # the small FP64 case
    "c0": dict(n=8192, nbins=42, precision="fp64", dt_myr=2.5, seed=0, run_steps=200,
               name="Test-1 Stromgren problem: 8192 interior vertices in the 13.2 kpc mirror box "
                    "+ sink shell, 42 bins, FP64, 200 steps of 2.5 Myr"),
}

# DRAM traffic of one k_step launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, the launch of step 305 of the headline run: state
# step 300, 5 warm-up steps), valid only for the kernel source it was taken
# on.
NCU_TRAFFIC = {"step_source_sha256": "b424a03402c3172cf34436d87d5c6bee069de5105d35d53741d0e9863789dfdf",
               "bytes_per_launch": 1079.232e6 + 392.197e6, "workload": "c1", "chem_fp32": False}


# ---------------------------------------------------------------------------
# distributed helpers (NCCL on GPUs; the CPU tests drive them with gloo)
# ---------------------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def dist_init(world: int, backend: str):
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist

        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
_CLK_FIELDS = ["timestamp", "index", "clocks.sm", "clocks.max.sm", "power.draw",
               "clocks_event_reasons.active", "clocks_event_reasons.hw_slowdown",
               "clocks_event_reasons.hw_thermal_slowdown",
               "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.samples = []
        self.proc = None
        self.gpu_index = gpu_index
        self.period_ms = period_ms
        self.t0 = self.t1 = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={','.join(_CLK_FIELDS)}", "--format=csv,noheader,nounits",
               f"-lms", str(self.period_ms), "-i", str(self.gpu_index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self._th = threading.Thread(target=self._read, daemon=True)
        self._th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, which: str):
        if which == "start":
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(self.period_ms / 1000.0 * 1.5)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for t, r in self.samples if self.t0 is not None and self.t0 <= t <= self.t1 + 0.05]
        if not rows:  # timed region shorter than one period: nearest sample
            rows = [min(self.samples, key=lambda s: abs(s[0] - (self.t0 or 0)))[1]] if self.samples else []
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[2]))
                smax = float(r[3])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[6:10]):
                if v.strip().lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def algorithmic_bytes_per_vertex(nbins: int, fp64: bool, mean_degree: float) -> float:
    """Bytes one vertex-step must move: its bin row read once and written once,
    y read and written (FP64), its adjacency (one 4-byte id per edge) and its
    constants (16 bytes)."""
    w = 8 if fp64 else 4
    return 2 * nbins * w + 16 + 4 * mean_degree + 16


def ballistic_bytes_per_vertex(mean_degree: float) -> float:
    """Bytes one vertex-step of ballistic transport must move: per edge, the
    FP32 packet on the in-edge read and the one on the out-edge written, the
    sender id and the packed straight set; y read and written and the
    constants (16 bytes each)."""
    return (4 + 4 + 4 + 4) * mean_degree + 16 + 16


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def kernel_source_sha() -> str:
    """sha256 of the step kernel's sources (sx_step.cu, then sx_step_common.cuh)."""
    h = hashlib.sha256()
    for f in ("sx_step.cu", "sx_step_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_0912_4273_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def make_problem(wl: dict, seed: int):
    from paper_0912_4273_gb300 import inputs as I

    return I.cached(I.stromgren_problem, wl["n"], seed=seed)


def chemistry_label(fp64: bool, chem_fp32: bool) -> str:
    if fp64:
        return "FP64 throughout"
    if chem_fp32:
        return "FP32 transport, FP32 subcycle rates with FP64 neutral fraction (the faster, less exact mode)"
    return "FP32 transport (compensated per-bin gathers), FP64 neutral fraction and recombination subcycling"


def run_ours(args, wl, rank, world, local_rank):
    import torch

    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    dist_init(world, "nccl")
    seed = wl["seed"] + rank
    prob = make_problem(wl, seed)
    bins = I.fibonacci_bins(wl["nbins"])
    dt = wl["dt_myr"] * I.MYR_S
    fp64 = wl["precision"] == "fp64"
    prec = S.SX_FP64 if fp64 else S.SX_FP32_TRANSPORT
    stream = torch.cuda.Stream(device)
    solver = S.Solver(bins, precision=prec, seed=seed, device=local_rank, stream=stream,
                      chem_fp32=args.chem_fp32).load(prob)
    n_int = int(prob.interior.sum())
    # untimed: the grid is advanced to the fixed state the timed steps start
    # from, then the warm-up steps
    state_step = min(args.state_step, max(wl["run_steps"] - args.steps - args.warmup, 0))
    solver.step(dt, state_step + args.warmup)
    solver.sync()
    t_first = state_step + args.warmup

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier(world, device)
    torch.cuda.synchronize(device)
    solver.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.mark("start")
    e0.record(stream)
    solver.step(dt, args.steps)
    e1.record(stream)
    e1.synchronize()
    clocks.mark("stop")
    torch.cuda.synchronize(device)
    barrier(world, device)
    ms = e0.elapsed_time(e1)
    info = solver.info
    solver.profile(False)
    clk = clocks.stop()
    max_ms = reduce_max(ms, world, device)
    value = aggregate(n_int * wl["nbins"] * args.steps, world, max_ms)
    kernel_ms = info["step_kernel_ms"] / max(info["step_kernel_launches"], 1)
    mean_deg = prob.nnz / prob.n
    per_vertex = algorithmic_bytes_per_vertex(wl["nbins"], fp64, mean_deg)
    bytes_launch = per_vertex * prob.n
    achieved = bytes_launch / (kernel_ms * 1e-3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    traffic = None
    if (NCU_TRAFFIC["step_source_sha256"] == kernel_source_sha() and NCU_TRAFFIC["workload"] == args.config
            and NCU_TRAFFIC.get("chem_fp32", False) == bool(args.chem_fp32)):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    budget = solver.budget
    solver.close()

    e2e = None
    if not args.no_e2e:  # whole job: every rank's replica, the slowest rank's time
        barrier(world, device)
        e2e = run_e2e(args, wl, prob, bins, dt, prec, seed, local_rank, stream)
        max_s = reduce_max(e2e["seconds"], world, device)
        e2e.update(value=aggregate(n_int * wl["nbins"] * e2e["steps"], world, max_s * 1e3),
                   seconds=max_s, h2d_bytes_per_step=e2e["h2d_bytes_per_step"] * world,
                   d2h_bytes_per_step=e2e["d2h_bytes_per_step"] * world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(wl, prob, bins, dt, seed)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
        "data": "synthetic (seeded Poisson-Delaunay Test-1 grid)",
        "config": {"workload": wl["name"] + f"; timed steps {t_first}..{t_first + args.steps - 1} "
                                            f"after an untimed advance to step {state_step}",
                   "state_step": state_step, "timed_steps": [t_first, t_first + args.steps],
                   "n_interior": n_int, "n_vertices": prob.n,
                   "nnz": prob.nnz, "nbins": wl["nbins"], "precision": chemistry_label(fp64, args.chem_fp32),
                   "chemistry": "f64" if (fp64 or not args.chem_fp32) else "f32 rates, f64 y",
                   "transport": "f64" if fp64 else "f32, compensated gathers",
                   "l2": (f"no flush: per-grid state {info['workspace_bytes'] / 1e9:.2f} GB > 129 MB L2"
                          if info["workspace_bytes"] > 129e6 else
                          f"no flush: per-grid state {info['workspace_bytes'] / 1e6:.0f} MB fits in the "
                          "129 MB L2 (a latency-bound case, not a bandwidth measurement)"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_step", "kernel_ms": kernel_ms,
                     "algorithmic_bytes_per_vertex": per_vertex,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if peaks else "fallback"},
        "clocks": clk,
        # the step kernels and one rotation launch per block of steps
        "gpu_launches": args.steps + -(-args.steps // S.SX_STEP_BLOCK),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "budget_residual": (budget["emitted"] - budget["absorbed"] - budget["escaped"]
                            - budget["in_flight"]) / max(budget["emitted"], 1e-300),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_e2e(args, wl, prob, bins, dt, prec, seed, local_rank, stream):
    """The whole job through the C ABI from pinned host buffers: load the grid
    (host->device), run the workload's full run (1000 steps for C1), every
    step reading the photon budget back into pinned memory (sx_step_budgets:
    queued behind its step, nothing waits), and read the neutral fraction at
    the end."""
    import torch

    from paper_0912_4273_gb300 import simplex as S

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()

    host = dict(pos=pinned(prob.pos), row_ptr=pinned(prob.row_ptr), col=pinned(prob.col),
                nH=pinned(prob.nH), volume=pinned(prob.volume), flags=pinned(prob.flags))
    y_out = pinned(np.zeros(prob.n))
    K = wl["run_steps"]
    budgets = pinned(np.zeros((K, 4)))
    h2d = sum(a.nbytes for a in host.values())
    solver = S.Solver(bins, precision=prec, seed=seed, device=local_rank, stream=stream,
                      chem_fp32=args.chem_fp32)
    nbytes = solver.workspace_bytes(prob.n, prob.nnz)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=torch.device("cuda", local_rank))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solver.load(workspace=ws, **host)
    for v, r in zip(prob.src_vertex, prob.src_rate):
        solver.add_source(int(v), float(r))
    solver.step_budgets(dt, K, budgets)
    S.sx_read_neutral_fraction(solver.ctx, y_out)
    t1 = time.perf_counter()
    assert budgets[-1, 0] > 0.0 and np.all(np.diff(budgets[:, 0]) > 0.0)  # every row arrived
    solver.close()
    n_int = int(prob.interior.sum())
    return {"value": n_int * wl["nbins"] * K / (t1 - t0), "unit": UNIT, "steps": K,
            "what": f"the whole {K}-step run from pinned host inputs: grid load, a budget read "
                    "per step, the neutral fraction at the end",
            "h2d_bytes_per_step": (h2d + 12 * len(prob.src_rate)) / K,
            "d2h_bytes_per_step": (y_out.nbytes + budgets.nbytes) / K,
            "seconds": t1 - t0}


def time_oracle(prob, bins, dt, seed, threads, budget_s, max_steps):
    """Oracle steps from the start of the run, timed one by one until
    budget_s seconds or max_steps steps; returns (steps, seconds, setup
    seconds).  The oracle sweeps every bin of every vertex, so a step costs
    the same at any state of the run."""
    import oracle as O

    t0 = time.perf_counter()
    sim = O.OracleSim(prob, O.Params(nbins=len(bins), seed=seed), bins, threads=threads)
    setup = time.perf_counter() - t0
    done, el = 0, 0.0
    while done < max_steps and el < budget_s:
        t0 = time.perf_counter()
        sim.step(dt, 1)
        el += time.perf_counter() - t0
        done += 1
    return done, el, setup


def run_cpu_baseline(wl, prob, bins, dt, seed):
    """The oracle (FP64, as it stands) on the same grid, on every host core
    (its threaded sweep, bit-identical to the serial one) and on one thread."""
    cores = os.cpu_count() or 1
    n_int = int(prob.interior.sum())
    steps_all, s_all, _ = time_oracle(prob, bins, dt, seed, cores, 12.0, 6)
    steps_one, s_one, _ = time_oracle(prob, bins, dt, seed, 1, 12.0, 3)
    v_all = n_int * wl["nbins"] * steps_all / s_all
    v_one = n_int * wl["nbins"] * steps_one / s_one
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps_all} FP64 oracle steps of the same grid from its start on {cores} "
                      f"threads (the oracle's cost per step does not depend on the state)",
            "single_thread": {"value": v_one, "cores": 1,
                              "sample": f"{steps_one} oracle steps, one thread"}}


def run_reference(args, wl, rank, world):
    """The oracle as the reference arm, on the workload's own grid: --warmup
    untimed steps, then --steps timed FP64 oracle steps on every host core
    (the threaded sweep).  Its cost per step does not depend on the state of
    the run, so the steps are taken from its start."""
    if rank != 0:
        return
    import oracle as O
    from paper_0912_4273_gb300 import inputs as I

    cores = os.cpu_count() or 1
    prob = make_problem(wl, wl["seed"])
    bins = I.fibonacci_bins(wl["nbins"])
    dt = wl["dt_myr"] * I.MYR_S
    sim = O.OracleSim(prob, O.Params(nbins=wl["nbins"], seed=wl["seed"]), bins, threads=cores)
    sim.step(dt, args.warmup)
    t0 = time.perf_counter()
    sim.step(dt, args.steps)
    el = time.perf_counter() - t0
    n_int = int(prob.interior.sum())
    value = n_int * wl["nbins"] * args.steps / el
    sample = (f"steps {args.warmup}..{args.warmup + args.steps - 1} of the FP64 oracle on the "
              f"workload's own grid ({prob.n} vertices, {wl['nbins']} bins), {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Poisson-Delaunay Test-1 grid)",
        "config": {"workload": wl["name"], "n_interior": n_int, "n_vertices": prob.n,
                   "nbins": wl["nbins"], "same_config": True,
                   "note": "the oracle sweeps every bin of every vertex: its cost per step does "
                           "not depend on the state, so it is timed from the start of the run"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# batched (many independent grids) and served (request stream) measurements
# ---------------------------------------------------------------------------
def _build_problem(recipe: str, n: int, seed: int):
    from paper_0912_4273_gb300 import inputs as I

    return I.cached(getattr(I, recipe), n, seed=seed)


def _build_problems(jobs):
    """(recipe name, n, seed) -> Problem for every job, the triangulations on
    up to 8 worker processes (spawned: they inherit no CUDA state), largest
    first."""
    import concurrent.futures as cf
    import multiprocessing as mp

    workers = min(len(jobs), os.cpu_count() or 1, 8)
    if workers <= 1:
        return [_build_problem(*j) for j in jobs]
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][1])
    out = [None] * len(jobs)
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        futs = {ex.submit(_build_problem, *jobs[i]): i for i in order}
        for f in cf.as_completed(futs):
            out[futs[f]] = f.result()
    return out


def _grid_pool(sizes, seed0=1000, recipe="stromgren_problem"):
    sizes = [int(n) for n in sizes]
    probs = _build_problems([(recipe, n, seed0 + i) for i, n in enumerate(sizes)])
    return dict(zip(sizes, probs))


def _sized_problem(base, nH, rate, box_over_rs=2.5):
    """A Test-1 problem on a pooled grid geometry rescaled to its own medium:
    the box is box_over_rs Stromgren radii across, with the source at the centre."""
    import copy

    from paper_0912_4273_gb300 import inputs as I

    rs = (3.0 * rate / (4.0 * math.pi * I.ALPHA_B * nH * nH)) ** (1.0 / 3.0)
    scale = box_over_rs * rs / base.box
    p = copy.copy(base)
    p.pos = base.pos * scale
    p.volume = base.volume * scale**3
    p.nH = np.full(base.n, nH)
    p.src_rate = np.array([rate])
    p.box = base.box * scale
    return p


def run_batched(args):
    """256 grids, sizes log-uniform in [4096, 262144], n_H log-uniform in
    [1e-4, 1e-2], one source each with rate log-uniform in [1e47, 1e49],
    42 bins, 500 steps of 4 t_rec / 500: one persistent launch per step for
    all grids (sx_batch_step) against one grid per launch sequence (sx_step)."""
    import torch

    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    rng = np.random.default_rng(args.seed)
    ngrids, steps = args.grids, args.batch_steps
    pool_sizes = np.unique(np.round(np.geomspace(4096, 262144, args.pool)).astype(int))
    pool = _grid_pool(pool_sizes)
    sizes = np.exp(rng.uniform(np.log(4096), np.log(262144), ngrids))
    pick = [int(pool_sizes[np.argmin(np.abs(np.log(pool_sizes) - np.log(n)))]) for n in sizes]
    nH = 10 ** rng.uniform(-4, -2, ngrids)
    rate = 10 ** rng.uniform(47, 49, ngrids)
    probs = [_sized_problem(pool[k], h, r) for k, h, r in zip(pick, nH, rate)]
    dts = [4.0 / (I.ALPHA_B * h) / steps for h in nH]
    bins = I.fibonacci_bins(42)
    st = torch.cuda.Stream()
    sol = [S.Solver(bins, seed=i, stream=st).load(p) for i, p in enumerate(probs)]
    batch = S.Batch(ngrids, stream=st)
    batch.step(sol, dts, 3)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(sol, dts, steps)
    for s in sol:
        s.sync()
    t_batch = time.perf_counter() - t0
    y_batch = [s.y for s in sol]
    for s in sol:
        s.close()
    batch.close()
    # one grid per launch sequence (sx_step, CUDA graphs), same work; loads
    # are outside the timed region as for the batch
    sol = [S.Solver(bins, seed=i, stream=st).load(p) for i, p in enumerate(probs)]
    for s, dt in zip(sol, dts):
        s.step(dt, 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s, dt in zip(sol, dts):
        s.step(dt, steps)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    y_plain = [s.y for s in sol]
    for s in sol:
        s.close()
    same = all(np.array_equal(a, b) for a, b in zip(y_batch, y_plain))
    nv = int(sum(int(p.interior.sum()) for p in probs))
    print(json.dumps({
        "mode": "batched", "grids": ngrids, "steps": steps, "interior_vertices": nv,
        "pool_geometries": len(pool_sizes), "nbins": 42,
        "batched": {"seconds": t_batch, "solves_per_s": ngrids / t_batch,
                    "updates_per_s": nv * 42 * steps / t_batch},
        "one_grid_per_launch": {"seconds": t_plain, "solves_per_s": ngrids / t_plain,
                                "updates_per_s": nv * 42 * steps / t_plain},
        "identical_results": same}), flush=True)


def run_served(args):
    """Serving (C4): a Poisson request stream (mean --rate per second) of
    solves with vertex counts log-uniform in [1e4, --serve-nmax] and, by coin
    flip, a uniform Test-1 medium (the C0/C1 generator) or the clumpy medium
    (the C2 generator: lognormal density, 16 sources); 42 or 84 bins; steps
    uniform in [100, --serve-steps-max].  Grids come from pools of prebuilt
    geometries (a fresh triangulation per request would take minutes at
    4e6 points); each request draws its own size (nearest pooled one),
    source rates, bins, steps and rotation seed.  Continuous batching (the
    server with every resident grid in every chunk, the headline, and with
    the least-remaining-work fill target of --serve-fills) against one
    request at a time on the plain path (sx_step with graphs); the results
    of every request are compared bit for bit across the policies."""
    import torch

    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import serve as SV

    rng = np.random.default_rng(args.seed)
    pool_sizes = np.unique(np.round(np.geomspace(1e4, args.serve_nmax, args.serve_pool)).astype(int))
    t_pool = time.perf_counter()
    sizes = [int(n) for n in pool_sizes]
    built = _build_problems([("stromgren_problem", n, 2000 + i) for i, n in enumerate(sizes)]
                            + [("clumpy_problem", n, 3000 + i) for i, n in enumerate(sizes)])
    uni = dict(zip(sizes, built[:len(sizes)]))
    clumpy = dict(zip(sizes, built[len(sizes):]))
    t_pool = time.perf_counter() - t_pool
    t = 0.0
    reqs = []
    for rid in range(args.requests):
        t += rng.exponential(1.0 / args.rate)
        n = np.exp(rng.uniform(np.log(1e4), np.log(args.serve_nmax)))
        k = int(pool_sizes[np.argmin(np.abs(np.log(pool_sizes) - np.log(n)))])
        nb = int(rng.choice([42, 84]))
        steps = int(rng.integers(100, args.serve_steps_max + 1))
        if rng.random() < 0.5:  # uniform Test-1 medium, box of 2.5 Stromgren radii
            nH = 1e-3
            rate = 10 ** rng.uniform(47.5, 49)
            prob = _sized_problem(uni[k], nH, rate)
            dt = 4.0 / (I.ALPHA_B * nH) / steps
            medium = "uniform"
        else:  # clumpy medium: its 16 sources with fresh log-uniform rates, 0.5 Myr steps
            import copy

            prob = copy.copy(clumpy[k])
            prob.src_rate = 10 ** rng.uniform(47, 49, len(prob.src_rate))
            dt = 0.5 * I.MYR_S
            medium = "clumpy"
        reqs.append(SV.Request(rid=rid, problem=prob, bins=I.fibonacci_bins(nb), steps=steps,
                               dt=dt, seed=rid, arrival=t))
        reqs[-1].medium = medium
    free, total = torch.cuda.mem_get_info()
    stats, results = {}, {}
    max_wait = SV.DEFAULT_MAX_WAIT_S if args.max_wait is None else (
        None if args.max_wait < 0 else args.max_wait)
    fills = [None if f in ("none", "every") else int(float(f)) for f in args.serve_fills.split(",")]
    for fill in fills:
        name = "continuous_batching" if fill == fills[0] else (
            "continuous_batching_every_grid" if fill is None else f"continuous_batching_fill_{fill}")
        be = SV.GpuBackend()
        srv = SV.Server(be, hbm_budget=int(0.6 * free), chunk_steps=args.chunk, fill_vertices=fill,
                        max_wait_s=max_wait)
        srv.run(reqs)
        be.close()
        stats[name] = dict(srv.stats(), fill_vertices=fill, max_wait_s=srv.max_wait,
                           chunk_steps=args.chunk)
        results[name] = {r.rid: r.y for r in reqs}
        for r in reqs:
            r.y = None
            r.status = "pending"
    st_p = SV.serve_one_at_a_time(reqs)
    same = all(np.array_equal(res[r.rid], r.y) for res in results.values() for r in reqs)
    work = float(sum(r.problem.n * len(r.bins) * r.steps for r in reqs))
    for v in list(stats.values()) + [st_p]:
        v["vertex_direction_updates_per_s"] = work / v["makespan_s"]
    print(json.dumps({"mode": "served", "requests": len(reqs), "rate_per_s": args.rate,
                      "n_range": [1e4, args.serve_nmax], "steps_range": [100, args.serve_steps_max],
                      "pool_geometries_per_medium": len(pool_sizes), "pool_build_s": t_pool,
                      "media": {m: sum(r.medium == m for r in reqs) for m in ("uniform", "clumpy")},
                      **stats, "one_at_a_time": st_p,
                      "speedup_solves_per_s": stats["continuous_batching"]["solves_per_s"]
                      / st_p["solves_per_s"],
                      "identical_results": same}), flush=True)


def run_transport(args):
    """Direction-conserving, ballistic and combined transport (tau_switch = 1,
    Sect. 5.1.3) on the C1 grid (Test 1, 2^20 interior vertices, 84 bins,
    FP32 transport, dt = 0.5 Myr): the step kernel's mean time over the same
    --steps after --warmup steps from a neutral start, timed with per-launch
    CUDA events.  Sect. 3.3 of the paper compares the three the same way."""
    import torch

    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    wl = WORKLOADS["c1"]
    prob = make_problem(wl, wl["seed"])
    bins = I.fibonacci_bins(wl["nbins"])
    dt = wl["dt_myr"] * I.MYR_S
    n_int = int(prob.interior.sum())
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    rows = {}
    for name, tp in (("direction_conserving", S.SX_TRANSPORT_DCT),
                     ("ballistic", S.SX_TRANSPORT_BALLISTIC),
                     ("combined_tau1", S.SX_TRANSPORT_COMBINED)):
        s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=wl["seed"], transport=tp,
                     tau_switch=1.0).load(prob)
        s.step(dt, args.warmup)
        s.sync()
        s.profile(True)
        s.step(dt, args.steps)
        info = s.info
        ms = info["step_kernel_ms"] / max(info["step_kernel_launches"], 1)
        b = s.budget
        y = s.y
        s.close()
        mean_deg = prob.nnz / prob.n
        if tp == S.SX_TRANSPORT_DCT:
            per_v = algorithmic_bytes_per_vertex(wl["nbins"], False, mean_deg)
        else:  # an edge packet read and written, sender id and straight set per edge; y, constants
            per_v = ballistic_bytes_per_vertex(mean_deg)
        gbs = per_v * prob.n / (ms * 1e-3) / 1e9
        rows[name] = {"step_kernel_ms": ms,
                      "vertex_steps_per_s": n_int / (ms * 1e-3),
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                   "frac": gbs / peak, "algorithmic_bytes_per_vertex": per_v},
                      "ionised_fraction": float(np.mean(y[prob.interior] < 0.5)),
                      "budget_residual": (b["emitted"] - b["absorbed"] - b["escaped"]
                                          - b["in_flight"]) / b["emitted"]}
        torch.cuda.synchronize()
    print(json.dumps({"mode": "transport", "workload": wl["name"], "steps": args.steps,
                      "warmup": args.warmup, **rows}), flush=True)


def shadow_depth_profile(p, y, max_cells: int = 20, behind_cells=None, slice_cells=None):
    """Ionised fraction (y < 0.5) of the vertices in the slab's geometric
    shadow, behind it and inside 0.85 r_S, by their distance in cells from the
    shadow cone's edge (bins of one cell); and the depth, in cells, of the
    first bin that is mostly neutral (the front's penetration).
    behind_cells: only vertices within that many cells behind the slab's far
    face; slice_cells: only vertices within that many cells of the source's
    z plane (a slice like the paper's figures)."""
    from paper_0912_4273_gb300 import inputs as I

    lo, hi = np.array(p.meta["slab_lo"]), np.array(p.meta["slab_hi"])
    c = p.pos[p.src_vertex[0]]
    d = p.pos - c
    rs = (3.0 * 5e48 / (4.0 * math.pi * I.ALPHA_B * 1e-6)) ** (1.0 / 3.0)
    cell = p.box / int(p.meta["n_interior"]) ** (1.0 / 3.0)
    near, far = lo[0] - c[0], hi[0] - c[0]
    x = d[:, 0]
    sel = (x > far + cell) & (np.linalg.norm(d, axis=1) < 0.85 * rs) & p.interior
    depth = np.minimum(0.5 * (hi[1] - lo[1]) * x / near - np.abs(d[:, 1]),
                       0.5 * (hi[2] - lo[2]) * x / near - np.abs(d[:, 2])) / cell
    sel &= depth > 0
    if behind_cells is not None:
        sel &= x < far + (1 + behind_cells) * cell
    if slice_cells is not None:
        sel &= np.abs(d[:, 2]) < slice_cells * cell
    prof, pen = [], None
    for k in range(max_cells):
        m = sel & (depth >= k) & (depth < k + 1)
        f = float((y[m] < 0.5).mean()) if m.any() else None
        prof.append(f)
        if pen is None and f is not None and f < 0.5:
            pen = k
    return prof, pen


def run_shadow(args):
    """Test 2 (Sect. 5.2): a point source and a slab 200 times denser than its
    surroundings, 500 Myr at dt = --shadow-dt Myr (0.5 by default), FP32
    transport, on the Test-1 grid at --shadow-res^3 points; 42 and 84 bins,
    and ballistic transport.  Reports, by depth in cells into the slab's
    shadow, the ionised fraction, and the penetration depth (the paper:
    about 5 cells at 64^3; 8 (84 bins) and 15 (42 bins) at 128^3), over the
    whole shadow out to 0.85 r_S and in a slice like the paper's figures
    (within 1.5 cells of the source's plane, 12 cells behind the slab)."""
    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    n = args.shadow_res ** 3
    t0 = time.perf_counter()
    p = I.cached(I.shadow_problem, n, seed=args.seed)
    t_grid = time.perf_counter() - t0
    out = {}
    dt_myr = args.shadow_dt
    steps = int(round(500.0 / dt_myr))
    for name, tp, nb in (("dct_84", S.SX_TRANSPORT_DCT, 84), ("dct_42", S.SX_TRANSPORT_DCT, 42),
                         ("ballistic", S.SX_TRANSPORT_BALLISTIC, 84)):
        s = S.Solver(I.fibonacci_bins(nb), precision=S.SX_FP32_TRANSPORT, seed=args.seed,
                     transport=tp).load(p)
        t0 = time.perf_counter()
        s.step(dt_myr * I.MYR_S, steps)
        y = s.y
        el = time.perf_counter() - t0
        s.close()
        prof, pen = shadow_depth_profile(p, y)
        sprof, spen = shadow_depth_profile(p, y, behind_cells=12, slice_cells=1.5)
        out[name] = {"penetration_cells": pen, "ionised_fraction_by_depth": prof,
                     "slice_penetration_cells": spen, "slice_ionised_fraction_by_depth": sprof,
                     "seconds": el}
    print(json.dumps({"mode": "shadow", "resolution": args.shadow_res, "n_vertices": p.n,
                      "dt_myr": dt_myr, "steps": steps, "grid_build_s": t_grid, **out}), flush=True)


def run_clumpy(args):
    """The clumpy medium (2^22 points by default, lognormal density on a 128^3
    mesh, 16 sources, 84 bins, FP32 transport, dt = 0.5 Myr) with the dynamic
    grid update of Sect. 2.1.4 every --update-every steps: vertices with
    y < 1e-3 whose mean edge is shorter than the mesh cell are removed
    (independent set), the cavities of the removed vertices re-triangulated
    on the host and the state carried over.  Reports the step kernel's throughput (per-launch CUDA
    events) and the cost of each update: marking on the device, local
    re-triangulation on the host (the library's native Bowyer-Watson per
    cavity, sx_remesh_remove), loading the new grid with the hand-over on
    the device."""
    import torch

    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import remesh as R
    from paper_0912_4273_gb300 import simplex as S

    n = args.clumpy_n
    t_gen = time.perf_counter()
    prob = I.cached(I.clumpy_problem, n, seed=args.seed)
    t_gen = time.perf_counter() - t_gen
    bins = I.fibonacci_bins(84)
    dt = 0.5 * I.MYR_S
    box = float(prob.box) if np.ndim(prob.box) == 0 else float(np.max(prob.box))
    min_spacing = box / 128.0
    n_start, nnz_start = prob.n, prob.nnz
    s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=args.seed).load(prob)
    s.step(dt, 3)  # warm-up
    s.sync()
    s.profile(True)
    done, upd_work = 3, 0.0
    updates = []
    while done < args.clumpy_steps:
        k = min(args.update_every - done % args.update_every, args.clumpy_steps - done)
        s.step(dt, k)
        upd_work += float(prob.interior.sum()) * len(bins) * k
        done += k
        if done % args.update_every or done >= args.clumpy_steps:
            continue
        s.sync()
        t0 = time.perf_counter()
        rem = s.mark_removal(1e-3, min_spacing)
        t1 = time.perf_counter()
        p2, o2n = R.remove_vertices(prob, rem)
        t2 = time.perf_counter()
        s.apply_update(p2, o2n)
        s.sync()
        t3 = time.perf_counter()
        updates.append({"step": done, "removed": int(len(rem)), "vertices_after": int(p2.n),
                        "mark_s": t1 - t0, "retriangulate_s": t2 - t1, "apply_s": t3 - t2})
        prob = p2
    s.sync()
    info = s.info
    ms = info["step_kernel_ms"] / max(info["step_kernel_launches"], 1)
    kernel_s = info["step_kernel_ms"] * 1e-3
    b = s.budget
    res = (b["emitted"] - b["absorbed"] - b["escaped"] - b["in_flight"]) / b["emitted"]
    s.close()
    print(json.dumps({
        "mode": "clumpy", "n_points": n, "n_vertices_start": n_start, "nnz_start": nnz_start,
        "grid_build_s": t_gen, "nbins": 84, "sources": 16, "steps": done,
        "update_every": args.update_every, "step_kernel_ms_mean": ms,
        "updates_per_s_step_kernel": upd_work / kernel_s if kernel_s > 0 else None,
        "grid_updates": updates, "budget_residual": res}), flush=True)


def run_accuracy(args):
    """The error of every result against the FP64 oracle on the small Test-1
    case (C0: 8192 interior vertices, 42 bins, 200 steps of 2.5 Myr), for
    each precision mode, with on-the-spot and with diffuse recombination
    radiation: neutral fraction per vertex (max and mean |dy|), each budget
    term and the photons in flight per vertex (relative to the emitted
    photons), and the ionised-volume radius."""
    import oracle as O
    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    prob = I.stromgren_problem(8192, seed=0)
    bins = I.fibonacci_bins(42)
    dt, steps = 2.5 * I.MYR_S, 200
    modes = (("fp64", S.SX_FP64, False), ("fp32_transport_fp64_chemistry", S.SX_FP32_TRANSPORT, False),
             ("fp32_transport_fp32_rates", S.SX_FP32_TRANSPORT, True))
    out = {}
    for rad, alpha_A in (("on_the_spot", 0.0), ("diffuse_case_A", 4.18e-13)):
        ref = O.OracleSim(prob, O.Params(nbins=42, seed=0, alpha_A=alpha_A), bins,
                          threads=os.cpu_count() or 1)
        ref.step(dt, steps)
        ry, rb, rph = ref.y, ref.budget, ref.photons()
        r_ref = O.ionised_radius_sphere(ry, prob.volume, prob.interior)
        for name, prec, f32 in modes:
            s = S.Solver(bins, precision=prec, seed=0, kappa=ref.kappa, chem_fp32=f32,
                         alpha_A=alpha_A).load(prob)
            s.step(dt, steps)
            y, b, ph = s.y, s.budget, s.photons()
            s.close()
            dy = np.abs(y - ry)
            out[f"{rad}/{name}"] = {
                "max_abs_dy": float(dy.max()), "mean_abs_dy": float(dy.mean()),
                "budget_rel_err": {k: abs(b[k] - rb[k]) / rb["emitted"] for k in rb},
                "photons_per_vertex_max_err_rel": float(np.abs(ph - rph).max() / rb["emitted"]),
                "ionised_radius_rel_err": abs(O.ionised_radius_sphere(y, prob.volume, prob.interior)
                                              / r_ref - 1.0)}
    print(json.dumps({"mode": "accuracy", "workload": WORKLOADS["c0"]["name"], "results": out}),
          flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(WORKLOADS), default="c1")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--state-step", type=int, default=300,
                    help="untimed steps before the warm-up (the state the timed steps start from)")
    ap.add_argument("--chem-fp32", action="store_true",
                    help="FP32 subcycle rates (the faster, less exact mode) instead of FP64 subcycles")
    ap.add_argument("--mode", choices=["step", "batched", "served", "clumpy", "transport", "shadow",
                                       "accuracy"], default="step")
    ap.add_argument("--shadow-res", type=int, default=128)
    ap.add_argument("--shadow-dt", type=float, default=0.5, help="shadow: time step in Myr")
    ap.add_argument("--clumpy-n", type=int, default=1 << 22)
    ap.add_argument("--clumpy-steps", type=int, default=200)
    ap.add_argument("--update-every", type=int, default=50)
    ap.add_argument("--grids", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--pool", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=6, help="served: pooled geometries per medium")
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--serve-nmax", type=float, default=4e6)
    ap.add_argument("--serve-steps-max", type=int, default=1000)
    ap.add_argument("--chunk", type=int, default=8)
    ap.add_argument("--serve-fills", default="none,131072",
                    help="served: fill targets in vertices to run (the first is the headline; "
                         "none = every resident grid in every chunk)")
    ap.add_argument("--max-wait", type=float, default=None,
                    help="served: seconds after which a request goes first (< 0: never)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    if args.mode == "batched":
        run_batched(args)
        return
    if args.mode == "served":
        run_served(args)
        return
    if args.mode == "clumpy":
        run_clumpy(args)
        return
    if args.mode == "transport":
        run_transport(args)
        return
    if args.mode == "shadow":
        run_shadow(args)
        return
    if args.mode == "accuracy":
        run_accuracy(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = dist_env()
    wl = WORKLOADS[args.config]
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    run_ours(args, wl, rank, world, local_rank)


if __name__ == "__main__":
    main()
