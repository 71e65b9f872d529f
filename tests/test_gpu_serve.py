"""The served form on the GPU: requests of different sizes and bin counts that
arrive while others run are batched together, and every result is identical
to the same request solved alone."""
import numpy as np
import pytest

from paper_0912_4273_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import serve as SV  # noqa: E402
from paper_0912_4273_gb300 import simplex as S  # noqa: E402


def _requests():
    rng = np.random.default_rng(3)
    out = []
    for rid in range(10):
        n = int(10 ** rng.uniform(2.5, 3.7))
        nb = 42 if rid % 3 else 84
        prob = I.stromgren_problem(n, seed=100 + rid)
        out.append(SV.Request(rid=rid, problem=prob, bins=I.fibonacci_bins(nb),
                              steps=int(rng.integers(10, 60)), dt=2.5 * I.MYR_S, seed=rid,
                              arrival=0.01 * rid))
    return out


@pytest.mark.parametrize("fill", [SV.DEFAULT_FILL_VERTICES, 4000])
def test_served_results_equal_solving_alone(fill):
    """With the default fill target every resident grid of a key shares each
    chunk; with 4000 vertices the chunks take subsets (least remaining work
    first), so grids pause and resume between chunks."""
    reqs = _requests()
    be = SV.GpuBackend()
    sizes = [be.footprint(r) for r in reqs]
    srv = SV.Server(be, hbm_budget=int(2.5 * max(sizes)), chunk_steps=5, fill_vertices=fill)
    done = srv.run(reqs)
    be.close()
    assert all(r.status == "done" for r in done)
    assert srv.peak_used <= srv.budget
    for r in done:
        s = S.Solver(r.bins, precision=r.precision, seed=r.seed).load(r.problem)
        s.step(r.dt, r.steps)
        assert np.array_equal(s.y, r.y), r.rid
        assert s.budget == r.budget
        s.close()
    st = srv.stats()
    assert st["solves"] == 10 and st["p99_s"] >= st["p50_s"]
