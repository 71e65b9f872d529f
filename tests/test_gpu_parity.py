"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (element by element):
  * SX_FP64: the same IEEE FP64 operations as the oracle's, some added in
    another fixed order (packets summed per new bin in edge order, N_in and
    the budget as reductions) and exp/expm1 from another library (1-2 ulp)
    -> |dy| <= 1e-9, budget 1e-9 relative.
  * SX_FP32_TRANSPORT: photons are rounded to FP32 at every hop (2^-24
    relative; every bin's packets summed with compensation), the chemistry
    in FP64 (or, with chem_fp32, its rates, subcycle lengths and
    exponentials in FP32 with y accumulated in FP64) -> |dy| <= 1e-4 per
    vertex and 1e-5 of the emitted photons for each budget term.
Routing decisions (association, straight table, bin remap) are integer on
both sides and therefore identical.
"""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I
from paper_0912_4273_gb300 import remesh as R

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import simplex as S  # noqa: E402

DT = 2.5 * I.MYR_S


def budget_err(b, rb):
    return max(abs(b[k] - rb[k]) for k in rb) / max(rb["emitted"], 1e-300)


@pytest.fixture(scope="module")
def c0():
    prob = I.stromgren_problem(8192, seed=0)
    bins = I.fibonacci_bins(42)
    ref = O.OracleSim(prob, O.Params(nbins=42, seed=0), bins)
    snaps = []
    for k in range(4):
        ref.step(DT, 50)
        snaps.append((ref.y.copy(), ref.budget, ref.I.sum(axis=1)))
    return prob, bins, ref, snaps


@pytest.mark.parametrize("variant", [4, 2])
@pytest.mark.parametrize("precision,chem_fp32,ytol,btol", [(S.SX_FP64, False, 1e-9, 1e-9),
                                                           (S.SX_FP32_TRANSPORT, False, 1e-4, 1e-5),
                                                           (S.SX_FP32_TRANSPORT, True, 1e-4, 1e-5)])
def test_c0_parity(c0, precision, chem_fp32, ytol, btol, variant):
    prob, bins, ref, snaps = c0
    s = S.Solver(bins, precision=precision, seed=0, kappa=ref.kappa, chem_fp32=chem_fp32).load(prob)
    s.variant = variant
    assert s.variant == variant
    for k in range(4):
        s.step(DT, 50)
        y_ref, b_ref, ph_ref = snaps[k]
        y = s.y
        assert np.abs(y - y_ref).max() <= ytol, (k, np.abs(y - y_ref).max())
        assert budget_err(s.budget, b_ref) <= btol
        ph = s.photons()
        assert np.abs(ph - ph_ref).max() <= btol * b_ref["emitted"]
    info = s.info
    assert info["step"] == 200
    assert info["capped"] == 0
    s.close()


def test_kappa_computed_on_device_matches_oracle(c0):
    prob, bins, ref, _ = c0
    s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT).load(prob)
    assert s.info["kappa"] == pytest.approx(ref.kappa, rel=1e-5)
    s.close()


@pytest.mark.parametrize("nbins", [6, 21, 32, 33, 63, 64, 65, 84, 128])
def test_bin_counts(nbins):
    prob = I.stromgren_problem(3000, seed=2)
    bins = I.fibonacci_bins(nbins)
    ref = O.OracleSim(prob, O.Params(nbins=nbins, seed=5), bins)
    ref.step(DT, 25)
    for precision, tol in ((S.SX_FP64, 1e-9), (S.SX_FP32_TRANSPORT, 1e-4)):
        s = S.Solver(bins, precision=precision, seed=5, kappa=ref.kappa).load(prob)
        s.step(DT, 25)
        assert np.abs(s.y - ref.y).max() <= tol
        assert budget_err(s.budget, ref.budget) <= (1e-9 if precision == S.SX_FP64 else 1e-5)
        s.close()


def test_deterministic_and_chunk_invariant(c0):
    prob, bins, ref, _ = c0
    out = []
    # blocks of rotation tables (SX_STEP_BLOCK steps per rotation launch)
    # split anywhere give the same steps; so do the timed launches
    for chunks, prof in (((60,), False), ((20, 40), False), ((1,) * 60, False),
                         ((17, 33, 10), True)):
        s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=0).load(prob)
        s.profile(prof)
        for c in chunks:
            s.step(DT, c)
        out.append((s.y, s.budget))
        s.close()
    for y, b in out[1:]:
        assert np.array_equal(y, out[0][0])
        assert b == out[0][1]


@pytest.mark.parametrize("steps", [20, 600])
def test_step_budgets_match_synchronous_reads(c0, steps):
    """sx_step_budgets queues a budget read behind every step (staged on the
    device, read back 256 steps at a time): the rows equal the budgets read
    synchronously after single steps, and the state equals sx_step's."""
    prob, bins, _, _ = c0
    a = S.Solver(bins, seed=0).load(prob)
    rows = []
    for _ in range(steps):
        a.step(DT, 1)
        b = a.budget
        rows.append([b["emitted"], b["absorbed"], b["escaped"], b["in_flight"]])
    c = S.Solver(bins, seed=0).load(prob)
    out = torch.zeros((steps, 4), dtype=torch.float64).pin_memory().numpy()
    c.step_budgets(DT, steps, out)
    c.sync()
    assert np.array_equal(np.array(rows), out)
    assert np.array_equal(a.y, c.y)
    assert a.budget == c.budget
    with pytest.raises(ValueError):
        c.step_budgets(DT, 3, np.zeros((2, 4)))
    a.close()
    c.close()


def test_transparent_medium_conserves_photons():
    p = np.random.default_rng(4).random((6000, 3))
    sink = np.any((p < 0.05) | (p > 0.95), axis=1)
    src = int(np.argmin(np.linalg.norm(p - 0.5, axis=1)))
    prob = I.point_process_problem(p, 1e-3, sink_mask=sink, sources=[(src, 1e50)])
    bins = I.fibonacci_bins(42)
    ref = O.OracleSim(prob, O.Params(nbins=42, sigma=0.0), bins)
    ref.step(1e13, 30)
    s = S.Solver(bins, sigma=0.0, kappa=ref.kappa).load(prob)
    s.step(1e13, 30)
    b = s.budget
    assert b["absorbed"] == 0.0
    assert b["emitted"] == pytest.approx(b["escaped"] + b["in_flight"], rel=1e-6)
    assert budget_err(b, ref.budget) <= 1e-5
    s.close()


def test_tiny_grid_and_no_sources():
    p = np.random.default_rng(0).random((9, 3))
    prob = I.point_process_problem(p, 1e-3, sources=[(0, 1e50)])
    bins = I.fibonacci_bins(21)
    ref = O.OracleSim(prob, O.Params(nbins=21), bins)
    ref.step(1e13, 7)
    s = S.Solver(bins, precision=S.SX_FP64, kappa=ref.kappa).load(prob)
    s.step(1e13, 7)
    assert np.abs(s.y - ref.y).max() <= 1e-9
    assert budget_err(s.budget, ref.budget) <= 1e-9
    s.close()
    # no sources: nothing changes from a neutral start
    prob.src_vertex = prob.src_vertex[:0]
    prob.src_rate = prob.src_rate[:0]
    s = S.Solver(bins).load(prob)
    s.step(1e13, 5)
    assert np.all(s.y == 1.0)
    assert all(v == 0.0 for v in s.budget.values())
    s.close()


def test_initial_ionisation_recombines_like_oracle():
    prob = I.stromgren_problem(2000, seed=3)
    bins = I.fibonacci_bins(42)
    y0 = np.random.default_rng(1).random(prob.n)
    ref = O.OracleSim(prob, O.Params(nbins=42, seed=3), bins, y0=y0)
    ref.step(DT, 10)
    s = S.Solver(bins, precision=S.SX_FP64, seed=3, kappa=ref.kappa).load(prob, y0=y0)
    s.step(DT, 10)
    assert np.abs(s.y - ref.y).max() <= 1e-9
    s.close()


def test_invalid_grids_are_rejected():
    prob = I.stromgren_problem(500, seed=0)
    bins = I.fibonacci_bins(42)
    s = S.Solver(bins)
    with pytest.raises(S.SimplexError) as e:
        s.step(DT, 1)
    assert e.value.code == S.SX_ESTATE
    # asymmetric: drop the first edge of vertex 0's row from the CSR
    rp = prob.row_ptr.copy()
    col = np.delete(prob.col, 0)
    rp[1:] -= 1
    with pytest.raises(S.SimplexError) as e:
        s.load(pos=prob.pos, row_ptr=rp, col=col, nH=prob.nH, volume=prob.volume, flags=prob.flags)
    assert e.value.code == S.SX_EINVAL and "symmetric" in str(e.value)
    # a row_ptr that decreases: refused on the host before any device work
    rp = prob.row_ptr.copy()
    rp[7] = rp[9] + 5
    with pytest.raises(S.SimplexError) as e:
        s.load(pos=prob.pos, row_ptr=rp, col=prob.col, nH=prob.nH, volume=prob.volume, flags=prob.flags)
    assert e.value.code == S.SX_EINVAL and "decrease" in str(e.value)
    # a non-sink star centre with more than SX_MAX_DEGREE neighbours
    n = 80
    pos = np.random.default_rng(0).normal(size=(n, 3))
    rows = [list(range(1, n))] + [[0] for _ in range(1, n)]
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col = np.concatenate(rows).astype(np.int32)
    with pytest.raises(S.SimplexError) as e:
        s.load(pos=pos, row_ptr=row_ptr, col=col, nH=np.ones(n), volume=np.ones(n),
               flags=np.zeros(n, np.uint8))
    assert e.value.code == S.SX_EINVAL and "degree" in str(e.value)
    # workspace too small
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.SimplexError) as e:
        s.load(prob, workspace=small)
    assert e.value.code == S.SX_ENOMEM
    s.close()


def test_batched_large_batch_takes_several_tiles_per_grab():
    """A batch whose tiles outnumber the persistent CTAs many times over
    (4 grids of 2^17 interior vertices: about 17k tiles, so several tiles per
    grab of the work queue) still matches each grid stepped alone."""
    bins = I.fibonacci_bins(42)
    probs = [I.cached(I.stromgren_problem, 1 << 17, seed=s) for s in (11, 12, 13, 14)]
    alone = []
    for p in probs:
        s = S.Solver(bins, seed=5).load(p)
        s.step(DT, 20)
        alone.append((s.y, s.budget))
        s.close()
    sol = [S.Solver(bins, seed=5).load(p) for p in probs]
    batch = S.Batch(max_grids=4)
    batch.step(sol, [DT] * 4, 20)
    for s, (y, b) in zip(sol, alone):
        assert np.array_equal(s.y, y)
        assert s.budget == b
        s.close()
    batch.close()


@pytest.mark.parametrize("variant", [4, 2])
def test_batched_step_equals_single_grid_steps(variant):
    """Grids stepped together in one persistent launch give bit-identical
    results to each grid stepped alone (every tile does the same arithmetic
    whichever CTA takes it), with the variant of the batch's first grid."""
    bins = I.fibonacci_bins(42)
    probs = [I.stromgren_problem(n, seed=s) for n, s in ((300, 1), (2048, 2), (5000, 3), (777, 4))]
    dts = [DT, 0.5 * DT, 2 * DT, DT]
    alone = []
    for p, dt in zip(probs, dts):
        s = S.Solver(bins, seed=7).load(p)
        s.variant = variant
        s.step(dt, 23)
        alone.append((s.y, s.budget, s.photons()))
        s.close()
    sol = [S.Solver(bins, seed=7).load(p) for p in probs]
    sol[0].variant = variant
    batch = S.Batch(max_grids=8)
    batch.step(sol, dts, 10)
    batch.step(sol, dts, 13)
    for s, (y, b, ph) in zip(sol, alone):
        assert s.info["step"] == 23
        assert np.array_equal(s.y, y)
        assert s.budget == b
        assert np.array_equal(s.photons(), ph)
        s.close()
    # mixed bin counts are refused
    other = S.Solver(I.fibonacci_bins(84)).load(probs[0])
    one = S.Solver(bins).load(probs[0])
    with pytest.raises(S.SimplexError) as e:
        batch.step([one, other], DT, 1)
    assert e.value.code == S.SX_EINVAL
    batch.close()


def test_graph_replay_on_a_stream_matches_direct_launches(c0):
    """On a non-default stream sx_step replays a captured CUDA graph of 16
    steps (one rotation launch for all 16, then their step launches); results
    are bit-identical to single-step launches."""
    prob, bins, ref, _ = c0
    st = torch.cuda.Stream()
    out = []
    for chunks in ((1,) * 40, (40,), (16, 3, 21)):
        s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=0, stream=st).load(prob)
        for c in chunks:
            s.step(DT, c)
        out.append((s.y, s.budget))
        s.close()
    for y, b in out[1:]:
        assert np.array_equal(y, out[0][0])
        assert b == out[0][1]
    # and the oracle agrees
    r = O.OracleSim(prob, O.Params(nbins=42, seed=0), bins)
    r.step(DT, 40)
    assert np.abs(out[1][0] - r.y).max() <= 1e-4


@pytest.mark.parametrize("precision,ytol,btol", [(S.SX_FP64, 1e-9, 1e-9),
                                                 (S.SX_FP32_TRANSPORT, 1e-4, 1e-5)])
def test_dynamic_update_parity(precision, ytol, btol):
    """Mark, hand over, re-triangulate, carry on: removal set, budget and
    neutral fractions agree with the oracle through the update."""
    prob = I.stromgren_problem(4096, seed=11)
    bins = I.fibonacci_bins(42)
    ref = O.OracleSim(prob, O.Params(nbins=42, seed=11), bins)
    kappa = ref.kappa
    s = S.Solver(bins, precision=precision, seed=11, kappa=kappa).load(prob)
    ref.step(DT, 80)
    s.step(DT, 80)
    _, _, ml = ref.tables()
    spacing = float(np.median(ml) * 1.2)
    rem = ref.mark_removal(1e-2, spacing)
    rem_gpu = s.mark_removal(1e-2, spacing)
    assert len(rem) > 10
    assert np.array_equal(rem, rem_gpu)
    # the oracle takes a full QHull rebuild of the survivors, the device the
    # local re-triangulation of the cavities: the same grid
    p2, o2n = I.survivor_problem(prob, rem)
    ref2 = ref.rebuild(rem, p2, o2n, params=O.Params(nbins=42, seed=11, kappa=kappa))
    p2l, o2nl = R.remove_vertices(prob, rem, allow_rebuild=False)
    assert np.array_equal(o2nl, o2n) and np.array_equal(p2l.col, p2.col)
    s.apply_update(p2l, o2nl)
    assert s.info["step"] == 80 and s.n == p2.n
    assert budget_err(s.budget, ref2.budget) <= btol
    assert np.abs(s.photons() - ref2.I.sum(axis=1)).max() <= btol * ref2.budget["emitted"]
    assert np.abs(s.y - ref2.y).max() <= ytol
    for _ in range(2):
        ref2.step(DT, 20)
        s.step(DT, 20)
        assert np.abs(s.y - ref2.y).max() <= ytol
        assert budget_err(s.budget, ref2.budget) <= btol
    # refused out of order: apply without a fresh mark
    with pytest.raises(S.SimplexError) as e:
        s.apply_update(p2, o2n)
    assert e.value.code == S.SX_ESTATE
    s.close()


@pytest.mark.parametrize("precision,ytol,btol", [(S.SX_FP64, 1e-9, 1e-9),
                                                 (S.SX_FP32_TRANSPORT, 1e-4, 1e-5)])
def test_clumpy_medium_with_16_sources(precision, ytol, btol):
    """Config-2 style medium (lognormal field, 16 sources) at a small size."""
    prob = I.clumpy_problem(12000, mesh=24, nsrc=16, seed=4)
    bins = I.fibonacci_bins(84)
    ref = O.OracleSim(prob, O.Params(nbins=84, seed=4), bins)
    s = S.Solver(bins, precision=precision, seed=4, kappa=ref.kappa).load(prob)
    for _ in range(3):
        ref.step(0.5 * I.MYR_S, 15)
        s.step(0.5 * I.MYR_S, 15)
        assert np.abs(s.y - ref.y).max() <= ytol
        assert budget_err(s.budget, ref.budget) <= btol
    assert s.info["nsources"] == 16
    s.close()


def test_autotune_leaves_the_state_and_keeps_a_variant(c0):
    """The autotuner times both step-kernel variants from the current state
    and restores it exactly; stepping on equals stepping with the chosen
    variant set by hand at the same point."""
    prob, bins, ref, snaps = c0
    s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=0, kappa=ref.kappa).load(prob)
    s.step(DT, 50)
    y, b, ph, st = s.y, s.budget, s.photons(), s.info["step"]
    r = s.autotune(DT, 4)
    # vertices per warp x row stride (42 bins: 44 or 48)
    assert sorted(zip(r["candidates"], r["strides"])) == [(2, 44), (2, 48), (4, 44), (4, 48)]
    assert r["variant"] in (2, 4) and r["stride"] in (44, 48)
    assert all(ms > 0 for ms in r["ms_per_step"])
    k = list(zip(r["candidates"], r["strides"])).index((r["variant"], r["stride"]))
    assert r["ms_per_step"][k] == min(r["ms_per_step"])
    assert s.variant == r["variant"] and s.bin_stride == r["stride"]
    assert np.array_equal(s.y, y) and s.budget == b and np.array_equal(s.photons(), ph)
    assert s.info["step"] == st
    s.step(DT, 50)
    u = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=0, kappa=ref.kappa).load(prob)
    u.step(DT, 50)
    u.variant = r["variant"]
    u.bin_stride = r["stride"]
    u.step(DT, 50)
    assert np.array_equal(s.y, u.y) and s.budget == u.budget
    y_ref, b_ref, _ = snaps[1]
    assert np.abs(s.y - y_ref).max() <= 1e-4
    assert budget_err(s.budget, b_ref) <= 1e-5
    with pytest.raises(S.SimplexError) as e:
        s.variant = 3
    assert e.value.code == S.SX_EINVAL
    s.close()
    u.close()


@pytest.mark.parametrize("nbins,strides", [(42, (44, 48)), (84, (84, 88)), (21, (24, 24))])
@pytest.mark.parametrize("precision", [S.SX_FP64, S.SX_FP32_TRANSPORT])
def test_bin_stride_changes_no_result(nbins, strides, precision, tmp_path):
    """The row stride of the stored photons (bin packing) is a layout
    choice: switching it mid-run, even twice, and across a checkpoint,
    leaves every result bit for bit as it was."""
    prob = I.stromgren_problem(3000, seed=4)
    bins = I.fibonacci_bins(nbins)
    a = S.Solver(bins, precision=precision, seed=2).load(prob)
    b = S.Solver(bins, precision=precision, seed=2).load(prob)
    assert a.bin_stride == strides[0]
    a.step(DT, 17)
    b.step(DT, 17)
    b.bin_stride = strides[1]
    assert b.bin_stride == strides[1]
    a.step(DT, 20)
    b.step(DT, 20)  # graphs, captured anew for the stride
    assert np.array_equal(a.y, b.y) and a.budget == b.budget and np.array_equal(a.photons(), b.photons())
    b.save(str(tmp_path / "s.ckpt"))
    c = S.Solver(bins, precision=precision, seed=2).restore(str(tmp_path / "s.ckpt"))
    assert c.bin_stride == strides[1]
    b.bin_stride = strides[0]
    for s in (a, b, c):
        s.step(DT, 9)
    for s in (b, c):
        assert np.array_equal(a.y, s.y) and a.budget == s.budget
    with pytest.raises(S.SimplexError):
        a.bin_stride = strides[1] + 4
    for s in (a, b, c):
        s.close()
