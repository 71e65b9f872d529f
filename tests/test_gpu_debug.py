"""The debug build (-DSX_DEBUG): the step kernels check every data-dependent
index (sender ids, packet bins, straight-set slots, reverse edges, the
ballistic in-edge lists) and count what is out of range instead of
touching it.  Direction-conserving, ballistic and combined solves and a
batch on grids with sinks, ragged tiles and the largest degree must find
nothing, and match the release build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
from paper_0912_4273_gb300 import inputs as I, simplex as S
from test_gpu_ballistic import _star
out = {}
for name, prob, nb, kw in (
        ("dct", I.stromgren_problem(3001, seed=2), 84, {}),
        ("dct128", I.stromgren_problem(1500, seed=3), 128, {}),
        ("ballistic", I.stromgren_problem(3001, seed=2), 42, dict(transport=S.SX_TRANSPORT_BALLISTIC)),
        ("combined", I.shadow_problem(16 ** 3, seed=1), 42, dict(transport=S.SX_TRANSPORT_COMBINED)),
        ("star", _star(), 42, dict(transport=S.SX_TRANSPORT_COMBINED))):
    for prec in (S.SX_FP64, S.SX_FP32_TRANSPORT):
        s = S.Solver(I.fibonacci_bins(nb), precision=prec, seed=1, **kw).load(prob)
        s.step(2.5 * I.MYR_S, 40)
        out[f"{name}_{prec}"] = [s.info["index_errors"], s.y.tolist()]
        s.close()
sols = [S.Solver(I.fibonacci_bins(42), seed=1).load(I.stromgren_problem(n, seed=n)) for n in (700, 2100)]
b = S.Batch(max_grids=4)
b.step(sols, 2.5 * I.MYR_S, 20)
out["batch"] = [sum(s.info["index_errors"] for s in sols), sols[0].y.tolist()]
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ, SIMPLEXGB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_finds_no_index_out_of_range():
    from paper_0912_4273_gb300 import build

    dbg = _run(build.build(debug=True))
    rel = _run(build.lib_path())
    for k, (errors, y) in dbg.items():
        assert errors == 0, k
        assert y == rel[k][1], k  # the checks change nothing when every index is in range
        assert rel[k][0] == 0
