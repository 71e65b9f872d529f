"""The host re-triangulation (Sect. 2.1.4) built with ThreadSanitizer and with
AddressSanitizer + UndefinedBehaviorSanitizer, on a grid large enough that
its passes and its cavity fill run on several threads: no report, and the
same grid as a full QHull rebuild of the survivors.  Skipped where g++ has
no sanitizer runtime."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0912_4273_gb300 import inputs as I
from test_remesh import _canon, _independent_interior

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def case(tmp_path_factory):
    # 2^16 points (about 450k tetrahedra, 1M edges) and 1200 cavities: the
    # passes over the arrays and the cavity fill all run on several threads
    p = I.stromgren_problem(1 << 16, seed=3)
    rem = _independent_interior(p, 1200, seed=1).astype(np.int32)
    d = tmp_path_factory.mktemp("remesh")
    np.array([p.n, len(p.simplices), len(rem)], dtype=np.int64).tofile(d / "hdr")
    np.ascontiguousarray(p.pos, dtype=np.float64).tofile(d / "pos")
    p.row_ptr.astype(np.int64).tofile(d / "row_ptr")
    p.col.astype(np.int32).tofile(d / "col")
    np.ascontiguousarray(p.simplices, dtype=np.int32).tofile(d / "tets")
    p.volume.astype(np.float64).tofile(d / "volume")
    rem.tofile(d / "removed")
    return p, rem, d


@pytest.mark.parametrize("sanitizer", ["thread", "address,undefined"])
def test_remesh_under_sanitizer(case, sanitizer, tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = tmp_path / "drv"
    src = [os.path.join(ROOT, "paper_0912_4273_gb300", "csrc", "sx_remesh.cpp"),
           os.path.join(ROOT, "tests", "remesh_driver.cpp")]
    cc = subprocess.run(["g++", "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer",
                         f"-fsanitize={sanitizer}", "-fno-sanitize-recover=all",
                         "-I", os.path.join(ROOT, "include"), *src, "-o", str(exe), "-lpthread"],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        pytest.skip(f"g++ cannot build with -fsanitize={sanitizer}: {cc.stderr[-300:]}")
    p, rem, d = case
    run = subprocess.run([str(exe), str(d)], capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, TSAN_OPTIONS="halt_on_error=1",
                                  ASAN_OPTIONS="halt_on_error=1", UBSAN_OPTIONS="halt_on_error=1"))
    assert run.returncode == 0, run.stderr[-3000:]
    assert "Sanitizer" not in run.stderr and "runtime error" not in run.stderr, run.stderr[-3000:]
    n, nnz, ntet = np.fromfile(d / "out_hdr", dtype=np.int64)
    full, old_of_new = I.survivor_problem(p, rem)
    assert n == full.n
    assert np.array_equal(np.fromfile(d / "out_old_of_new", dtype=np.int32), old_of_new)
    assert np.array_equal(np.fromfile(d / "out_row_ptr", dtype=np.int64), full.row_ptr)
    assert np.array_equal(np.fromfile(d / "out_col", dtype=np.int32), full.col)
    np.testing.assert_allclose(np.fromfile(d / "out_volume"), full.volume, rtol=1e-11, atol=0)
    tets = np.fromfile(d / "out_tets", dtype=np.int32).reshape(-1, 4)
    assert len(tets) == ntet and np.array_equal(_canon(tets), _canon(full.simplices))
