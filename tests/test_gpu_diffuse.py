"""Diffuse recombination radiation on the GPU (Sect. 2.2.1, 4.5) against the
FP64 oracle, element by element.

With alpha_A > 0 the cells recombine at case A, and the ground-level share
(alpha_A - alpha_B) / alpha_A of each step's recombinations is emitted in
the next step: an equal share in every bin after the sources' photons, or,
at a ballistic vertex, with its own photons to all its neighbours.  The
neutral fractions, the photons in flight towards every vertex and the
budget (whose emitted photons include the diffuse ones) are compared over
many steps, in direction-conserving, ballistic and combined transport, at the
tolerances of the plain runs: FP64 1e-9; FP32 transport 1e-4 in y and 1e-5 of
the emitted photons per budget term.
"""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import simplex as S  # noqa: E402

ALPHA_A = 4.18e-13  # case A at 1e4 K (cm^3/s)
DT = 2.5 * I.MYR_S
DCT, BAL, COMB = S.SX_TRANSPORT_DCT, S.SX_TRANSPORT_BALLISTIC, S.SX_TRANSPORT_COMBINED


@pytest.fixture(scope="module")
def grid():
    return I.stromgren_problem(4096, seed=8)


def _budget_err(b, rb):
    return max(abs(b[k] - rb[k]) for k in rb) / rb["emitted"]


@pytest.mark.parametrize("transport,tau_switch,nbins", [(DCT, 1.0, 42), (DCT, 1.0, 84),
                                                        (BAL, 0.0, 42), (COMB, 1.0, 42)])
@pytest.mark.parametrize("precision,chem_fp32,ytol,btol", [(S.SX_FP64, False, 1e-9, 1e-9),
                                                           (S.SX_FP32_TRANSPORT, False, 1e-4, 1e-5),
                                                           (S.SX_FP32_TRANSPORT, True, 1e-4, 1e-5)])
def test_parity_with_oracle(grid, transport, tau_switch, nbins, precision, chem_fp32, ytol, btol):
    bins = I.fibonacci_bins(nbins)
    p = O.Params(nbins=nbins, seed=8, transport=transport, tau_switch=tau_switch, alpha_A=ALPHA_A)
    ref = O.OracleSim(grid, p, bins)
    s = S.Solver(bins, precision=precision, seed=8, kappa=ref.kappa, transport=transport,
                 tau_switch=tau_switch, alpha_A=ALPHA_A, chem_fp32=chem_fp32).load(grid)
    for steps in (1, 16, 23, 40):  # 80 steps: graphs and direct launches
        ref.step(DT, steps)
        s.step(DT, steps)
        assert np.abs(s.y - ref.y).max() <= ytol
        rb = ref.budget
        assert _budget_err(s.budget, rb) <= btol, (s.budget, rb)
        assert np.abs(s.photons() - ref.photons()).max() <= btol * rb["emitted"]
    # the cells did re-emit: the emitted photons exceed the source's
    assert ref.diffuse()[1] > 0.05 * ref.budget["emitted"]
    assert s.budget["emitted"] > grid.src_rate.sum() * DT * 80 * 1.05
    s.close()


def test_diffuse_radiation_off_is_the_on_the_spot_kernel(grid):
    """alpha_A = 0 runs the kernel as before, bit for bit with a context
    created without the field set (the default)."""
    bins = I.fibonacci_bins(42)
    out = []
    for kw in (dict(), dict(alpha_A=0.0)):
        s = S.Solver(bins, seed=2, **kw).load(grid)
        s.step(DT, 30)
        out.append((s.y, s.budget))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_deterministic_and_checkpointed(grid, tmp_path):
    """Reruns give the same bits, and a checkpoint taken mid-run (with the
    cells' pending photons) continues bit-identically."""
    bins = I.fibonacci_bins(42)
    a = S.Solver(bins, seed=4, alpha_A=ALPHA_A).load(grid)
    a.step(DT, 37)
    a.save(str(tmp_path / "d.ckpt"))
    a.step(DT, 25)
    b = S.Solver(bins, seed=4, alpha_A=ALPHA_A).restore(str(tmp_path / "d.ckpt"))
    b.step(DT, 25)
    c = S.Solver(bins, seed=4, alpha_A=ALPHA_A).load(grid)
    c.step(DT, 62)
    for x in (b, c):
        assert np.array_equal(a.y, x.y) and a.budget == x.budget
    for x in (a, b, c):
        x.close()


def test_grid_update_refuses_diffuse_radiation(grid):
    s = S.Solver(I.fibonacci_bins(42), alpha_A=ALPHA_A).load(grid)
    s.step(DT, 3)
    with pytest.raises(S.SimplexError) as e:
        s.mark_removal(1e-3, 1e30)
    assert e.value.code == S.SX_EINVAL
    s.close()


def test_bad_alpha_A_is_refused():
    with pytest.raises(S.SimplexError):
        S.Solver(I.fibonacci_bins(42), alpha_A=1e-13)  # below alpha_B
