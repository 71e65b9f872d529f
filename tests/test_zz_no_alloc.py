"""sx_kappa_noalloc: kappa for callers that cannot allocate device memory.

Such a caller cannot provide the device workspace that sx_load_grid needs,
so it gets kappa from an entry point whose device scratch is a fixed array
inside the library.  Its value must equal the one sx_load_grid computes for
the same grid, on every call (the scratch keeps the previous call's contents).
This file is collected last so that a failure here stops a run only after
every other test has run.
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

KAPPA_RTOL = 1e-12  # same kernels, same inputs, same order of operations


@pytest.mark.parametrize("nbins", [42, 84])
def test_kappa_noalloc_matches_load_grid_twice(nbins):
    prob = I.stromgren_problem(8192, seed=0)  # 12.4k vertices, ~190k edges: within the limits
    assert prob.n <= S.SX_NOALLOC_MAX_VERTICES and prob.nnz <= S.SX_NOALLOC_MAX_EDGES
    bins = I.fibonacci_bins(nbins)
    s = S.Solver(bins).load(prob)
    k_ref = s.info["kappa"]
    s.close()
    for _ in range(2):
        k = S.sx_kappa_noalloc(prob.n, prob.pos, prob.row_ptr, prob.col, prob.flags, bins)
        assert k == pytest.approx(k_ref, rel=KAPPA_RTOL)
    # and the oracle's kappa (FP64 sums of the FP32 per-vertex ratios: 1e-5)
    assert k == pytest.approx(O.OracleSim(prob, O.Params(nbins=nbins), bins).kappa, rel=1e-5)
    # a different grid in between, then the first again: no state leaks across calls
    small = I.stromgren_problem(1000, seed=5)
    s = S.Solver(bins).load(small)
    k_small = s.info["kappa"]
    s.close()
    assert S.sx_kappa_noalloc(small.n, small.pos, small.row_ptr, small.col, small.flags,
                              bins) == pytest.approx(k_small, rel=KAPPA_RTOL)
    assert S.sx_kappa_noalloc(prob.n, prob.pos, prob.row_ptr, prob.col, prob.flags,
                              bins) == pytest.approx(k_ref, rel=KAPPA_RTOL)


def test_kappa_noalloc_refuses_grids_beyond_its_scratch():
    n = S.SX_NOALLOC_MAX_VERTICES + 1
    with pytest.raises(S.SimplexError) as e:
        S.sx_kappa_noalloc(n, np.zeros((n, 3)), np.zeros(n + 1, np.int64), np.zeros(0, np.int32),
                           np.zeros(n, np.uint8), I.fibonacci_bins(42))
    assert e.value.code == S.SX_EINVAL and "SX_NOALLOC_MAX_VERTICES" in str(e.value)
    n = 100
    rp = np.zeros(n + 1, np.int64)
    rp[-1] = S.SX_NOALLOC_MAX_EDGES + 1
    with pytest.raises(S.SimplexError) as e:
        S.sx_kappa_noalloc(n, np.zeros((n, 3)), rp, np.zeros(rp[-1], np.int32),
                           np.zeros(n, np.uint8), I.fibonacci_bins(42))
    assert e.value.code == S.SX_EINVAL
