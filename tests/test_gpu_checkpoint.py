"""Checkpoints: a grid saved mid-run and restored into a fresh context steps
on to results bit-identical to the run that was not interrupted (tables,
neutral fractions, photons in flight, routing, budget, sources and step
counters all come back), also right after a dynamic grid update."""
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


def state(s):
    return s.y, s.budget, s.photons(), s.info["step"]


def same(a, b):
    return (np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
            and a[3] == b[3])


@pytest.mark.parametrize("precision", [S.SX_FP64, S.SX_FP32_TRANSPORT])
def test_restore_continues_bit_identically(tmp_path, precision):
    prob = I.stromgren_problem(3000, seed=4)
    bins = I.fibonacci_bins(42)
    s = S.Solver(bins, precision=precision, seed=9).load(prob)
    s.step(DT, 31)
    path = str(tmp_path / "run.sxck")
    s.save(path)
    assert S.sx_checkpoint_info(path) == (prob.n, int(prob.row_ptr[-1]))
    s.step(DT, 23)
    want = state(s)
    kappa = s.info["kappa"]
    # a fresh context with another seed and kappa: the checkpoint's are used
    t = S.Solver(bins, precision=precision, seed=1, kappa=0.5).restore(path)
    assert t.info["step"] == 31 and t.n == prob.n and t.info["kappa"] == kappa
    t.step(DT, 23)
    assert same(state(t), want)
    # restoring again rewinds
    t.restore(path)
    t.step(DT, 23)
    assert same(state(t), want)
    s.close()
    t.close()


def test_restore_after_a_grid_update(tmp_path):
    """Saved right after sx_grid_update_apply: the carried photons wait in the
    incoming field and the budget carries the replaced grid's terms."""
    prob = I.stromgren_problem(4096, seed=11)
    bins = I.fibonacci_bins(42)
    s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=11).load(prob)
    s.step(DT, 80)
    ml = O.OracleSim(prob, O.Params(nbins=42, seed=11), bins).tables()[2]
    rem = s.mark_removal(1e-2, float(np.median(ml) * 1.2))
    assert len(rem) > 10
    with pytest.raises(S.SimplexError) as e:  # a marked update must be applied first
        s.save(str(tmp_path / "x.sxck"))
    assert e.value.code == S.SX_ESTATE
    p2, o2n = I.survivor_problem(prob, rem)
    s.apply_update(p2, o2n)
    path = str(tmp_path / "upd.sxck")
    s.save(path)
    s.step(DT, 17)
    want = state(s)
    t = S.Solver(bins, precision=S.SX_FP32_TRANSPORT).restore(path)
    t.step(DT, 17)
    assert same(state(t), want)
    s.close()
    t.close()


def test_restore_refuses_other_bins_and_non_checkpoints(tmp_path):
    prob = I.stromgren_problem(1000, seed=2)
    s = S.Solver(I.fibonacci_bins(42)).load(prob)
    s.step(DT, 3)
    path = str(tmp_path / "a.sxck")
    s.save(path)
    other = S.Solver(I.fibonacci_bins(21))
    with pytest.raises(S.SimplexError) as e:
        other.restore(path)
    assert e.value.code == S.SX_EINVAL
    bad = tmp_path / "not.sxck"
    bad.write_bytes(b"hello")
    with pytest.raises(S.SimplexError) as e:
        s.restore(str(bad))
    assert e.value.code == S.SX_EINVAL
    # the file sx_save wrote verifies; a copy with one byte changed in its
    # body is refused before the context is touched, which keeps its grid
    S.sx_checkpoint_verify(path)
    data = bytearray(open(path, "rb").read())
    data[len(data) // 2] ^= 0x10
    damaged = tmp_path / "damaged.sxck"
    damaged.write_bytes(bytes(data))
    y = s.y
    with pytest.raises(S.SimplexError) as e:
        s.restore(str(damaged))
    assert e.value.code == S.SX_EINVAL and "damaged" in str(e.value)
    assert np.array_equal(s.y, y)
    s.close()
    other.close()


def test_library_fibonacci_bins():
    """NULL bin directions: the library's own Fibonacci lattice, which agrees
    with the unordered lattice of the input generator (same formula)."""
    prob = I.stromgren_problem(2000, seed=6)
    a = S.Solver(42, precision=S.SX_FP64, seed=2).load(prob)
    b = S.Solver(I.fibonacci_bins(42, ordered=False), precision=S.SX_FP64, seed=2).load(prob)
    a.step(DT, 20)
    b.step(DT, 20)
    assert np.abs(a.y - b.y).max() <= 1e-9
    a.close()
    b.close()
