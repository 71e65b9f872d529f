"""The shadowing test (Test 2, Sect. 5.2) on the GPU: element-wise parity with
the oracle on the slab grid (its 200x density contrast drives the chemistry
to large optical depths), and at 64^3 the shadow: the shadowed region stays
mostly neutral away from its edge while the mirror region is ionised, and
direction-conserving transport shadows better than ballistic transport."""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import simplex as S  # noqa: E402
from test_oracle_shadow import shadow_regions  # noqa: E402


@pytest.mark.parametrize("transport", [S.SX_TRANSPORT_DCT, S.SX_TRANSPORT_COMBINED])
@pytest.mark.parametrize("precision,ytol,btol", [(S.SX_FP64, 1e-9, 1e-9),
                                                 (S.SX_FP32_TRANSPORT, 1e-4, 1e-5)])
def test_parity_on_the_slab_grid(transport, precision, ytol, btol):
    p = I.cached(I.shadow_problem, 32 ** 3, seed=0)
    bins = I.fibonacci_bins(42)
    ref = O.OracleSim(p, O.Params(nbins=42, seed=0, transport=transport), bins)
    s = S.Solver(bins, precision=precision, seed=0, kappa=ref.kappa, transport=transport).load(p)
    ref.step(5 * I.MYR_S, 40)
    s.step(5 * I.MYR_S, 40)
    assert np.abs(s.y - ref.y).max() <= ytol
    rb = ref.budget
    assert max(abs(s.budget[k] - rb[k]) for k in rb) <= btol * rb["emitted"]
    s.close()


def test_shadow_at_64_cubed():
    p = I.cached(I.shadow_problem, 64 ** 3, seed=0)
    shadow, mirror = shadow_regions(p, 6)
    assert shadow.sum() > 1000
    ion = {}
    for tp, nb in ((S.SX_TRANSPORT_DCT, 84), (S.SX_TRANSPORT_DCT, 42), (S.SX_TRANSPORT_BALLISTIC, 84)):
        s = S.Solver(I.fibonacci_bins(nb), seed=0, transport=tp).load(p)
        s.step(0.5 * I.MYR_S, 1000)  # 500 Myr
        y = s.y
        s.close()
        assert (y[mirror] < 0.5).mean() > 0.95
        ion[(tp, nb)] = (y[shadow] < 0.5).mean()
    # the front penetrates about 5 cells into the shadow at 64^3 (Sect. 5.2):
    # 6 cells inside the shadow's edge the medium is mostly neutral
    assert ion[(S.SX_TRANSPORT_DCT, 84)] < 0.5
    assert ion[(S.SX_TRANSPORT_DCT, 42)] < 0.5
    assert ion[(S.SX_TRANSPORT_BALLISTIC, 84)] > ion[(S.SX_TRANSPORT_DCT, 84)] + 0.05
