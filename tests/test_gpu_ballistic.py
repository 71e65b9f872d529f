"""Ballistic and combined transport on the GPU (Sect. 2.2.2, 2.2.4) against
the FP64 oracle, element by element: neutral fractions, photons in flight per
vertex and the photon budget, through the same launches as direction-
conserving transport (the step kernel with thick vertices)."""
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
