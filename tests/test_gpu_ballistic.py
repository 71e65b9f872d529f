"""Ballistic and combined transport on the GPU (Sect. 2.2.2, 2.2.4) against
the FP64 oracle, element by element: neutral fractions, photons in flight per
vertex and the photon budget, through the same launches as direction-
conserving transport (the step kernel with thick vertices); ballistic
transport alone has a kernel of its own, which must step exactly as the
combined kernel does when every vertex is thick."""
import math

import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import simplex as S  # noqa: E402

DT = 2.5 * I.MYR_S
BAL, COMB = S.SX_TRANSPORT_BALLISTIC, S.SX_TRANSPORT_COMBINED


@pytest.fixture(scope="module")
def grid():
    return I.stromgren_problem(4096, seed=5)


def _budget_err(b, rb):
    return max(abs(b[k] - rb[k]) for k in rb) / rb["emitted"]


@pytest.mark.parametrize("nbins", [42, 84])
@pytest.mark.parametrize("transport,tau_switch", [(BAL, 0.0), (COMB, 1.0), (COMB, 0.05)])
@pytest.mark.parametrize("precision,ytol,btol", [(S.SX_FP64, 1e-9, 1e-9),
                                                 (S.SX_FP32_TRANSPORT, 1e-4, 1e-5)])
def test_parity_with_oracle(grid, nbins, transport, tau_switch, precision, ytol, btol):
    bins = I.fibonacci_bins(nbins)
    ref = O.OracleSim(grid, O.Params(nbins=nbins, seed=5, transport=transport, tau_switch=tau_switch),
                      bins)
    s = S.Solver(bins, precision=precision, seed=5, kappa=ref.kappa, transport=transport,
                 tau_switch=tau_switch).load(grid)
    for steps in (3, 17, 20):  # 40 steps: graphs and direct launches, modes changing as the front moves
        ref.step(DT, steps)
        s.step(DT, steps)
        assert np.abs(s.y - ref.y).max() <= ytol
        rb = ref.budget
        assert _budget_err(s.budget, rb) <= btol
        assert np.abs(s.photons() - ref.photons()).max() <= btol * rb["emitted"]
    thick = ref.ballistic()[2]
    if transport == COMB:
        assert 0 < thick.sum() < grid.n  # both modes present
    s.close()


@pytest.mark.parametrize("precision", [S.SX_FP64, S.SX_FP32_TRANSPORT])
def test_ballistic_kernel_is_combined_with_every_vertex_thick(grid, precision):
    """tau_switch = 0 makes every cell thick (y tau_max >= 0), so the combined
    kernel's ballistic tiles run the same step as the ballistic kernel:
    neutral fractions and photons in flight bit for bit; the budget to
    rounding (a sink sums what reaches it in another order)."""
    bins = I.fibonacci_bins(84)
    out = []
    for tp in (BAL, COMB):
        s = S.Solver(bins, precision=precision, seed=4, transport=tp, tau_switch=0.0).load(grid)
        for steps in (1, 16, 23):
            s.step(DT, steps)
            out.append((tp, s.y, s.photons(), s.budget))
        s.close()
    for (_, y0, p0, b0), (_, y1, p1, b1) in zip(out[:3], out[3:]):
        assert np.array_equal(y0, y1)
        assert np.array_equal(p0, p1)
        assert _budget_err(b0, b1) <= 1e-12


def test_combined_with_infinite_switch_is_the_direction_conserving_kernel(grid):
    bins = I.fibonacci_bins(42)
    out = []
    for kw in (dict(), dict(transport=COMB, tau_switch=math.inf)):
        s = S.Solver(bins, seed=2, **kw).load(grid)
        s.step(DT, 30)
        out.append((s.y, s.budget, s.photons()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


def test_deterministic_and_chunk_invariant(grid):
    bins = I.fibonacci_bins(42)
    st = torch.cuda.Stream()
    out = []
    for chunks in ((40,), (16, 3, 21), (1,) * 40):
        s = S.Solver(bins, seed=1, transport=COMB, tau_switch=1.0, stream=st).load(grid)
        for c in chunks:
            s.step(DT, c)
        out.append((s.y, s.budget))
        s.close()
    for y, b in out[1:]:
        assert np.array_equal(y, out[0][0]) and b == out[0][1]


def test_direction_conserving_only_calls_are_refused(grid, tmp_path):
    bins = I.fibonacci_bins(42)
    s = S.Solver(bins, transport=BAL).load(grid)
    s.step(DT, 2)
    for call in (lambda: s.mark_removal(1e-3, 1.0), lambda: s.save(str(tmp_path / "x")),
                 lambda: setattr(s, "variant", 4)):
        with pytest.raises(S.SimplexError) as e:
            call()
        assert e.value.code == S.SX_EINVAL and "direction-conserving" in str(e.value)
    batch = S.Batch(max_grids=2)
    with pytest.raises(S.SimplexError) as e:
        batch.step([s], DT, 1)
    assert e.value.code == S.SX_EINVAL
    batch.close()
    s.close()
    with pytest.raises(S.SimplexError):
        S.Solver(bins, transport=7)


def _star(narms=64):
    """A source at the centre with narms arms of two vertices (inner at 1 kpc,
    outer at 2 kpc, the outer ones sinks): the centre has the largest degree
    a non-sink vertex may have."""
    d = I.fibonacci_bins(narms)
    pos = np.concatenate([np.zeros((1, 3)), d * I.KPC_CM, 2 * d * I.KPC_CM])
    n = len(pos)
    nbr = [list(range(1, narms + 1))]
    nbr += [[0, narms + i] for i in range(1, narms + 1)]
    nbr += [[i] for i in range(1, narms + 1)]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(x) for x in nbr])
    col = np.concatenate([np.sort(x) for x in nbr]).astype(np.int32)
    flags = np.zeros(n, dtype=np.uint8)
    flags[narms + 1:] = I.FLAG_SINK
    return I.Problem(pos=pos, row_ptr=row_ptr, col=col, nH=np.full(n, 1e-3),
                     volume=np.full(n, (0.5 * I.KPC_CM) ** 3), flags=flags,
                     src_vertex=np.array([0], dtype=np.int32), src_rate=np.array([5e48]),
                     box=4 * I.KPC_CM, meta=dict(kind="star"))


@pytest.mark.parametrize("transport", [S.SX_TRANSPORT_DCT, BAL, COMB])
@pytest.mark.parametrize("precision,ytol,btol", [(S.SX_FP64, 1e-9, 1e-9),
                                                 (S.SX_FP32_TRANSPORT, 1e-4, 1e-5)])
def test_largest_degree_and_empty_straight_sets(transport, precision, ytol, btol):
    """The centre (degree 64) fills a thick vertex's 64 in-edge slots and both
    halves of the warp in the send; an inner arm vertex sends nothing back
    towards the centre (its only other edge is beyond 90 degrees of the
    incoming direction, so photons from outside escape)."""
    prob = _star()
    assert np.diff(prob.row_ptr)[0] == 64
    bins = I.fibonacci_bins(42)
    ref = O.OracleSim(prob, O.Params(nbins=42, seed=4, transport=transport, tau_switch=1.0), bins)
    s = S.Solver(bins, precision=precision, seed=4, kappa=ref.kappa, transport=transport,
                 tau_switch=1.0).load(prob)
    for steps in (1, 2, 9):
        ref.step(DT, steps)
        s.step(DT, steps)
        assert np.abs(s.y - ref.y).max() <= ytol
        assert _budget_err(s.budget, ref.budget) <= btol
        assert np.abs(s.photons() - ref.photons()).max() <= btol * ref.budget["emitted"]
    s.close()


@pytest.mark.parametrize("nbins", [21, 128])
def test_mask_word_counts(grid, nbins):
    """One and four mask words (21 and 128 bins) through the thick-vertex
    paths of combined transport, FP64."""
    bins = I.fibonacci_bins(nbins)
    ref = O.OracleSim(grid, O.Params(nbins=nbins, seed=5, transport=COMB, tau_switch=1.0), bins)
    s = S.Solver(bins, precision=S.SX_FP64, seed=5, kappa=ref.kappa, transport=COMB,
                 tau_switch=1.0).load(grid)
    ref.step(DT, 25)
    s.step(DT, 25)
    assert np.abs(s.y - ref.y).max() <= 1e-9
    assert _budget_err(s.budget, ref.budget) <= 1e-9
    s.close()
