"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/simplexgb.h declares (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0912_4273_gb300 import build

    return build.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "simplexgb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sx_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sx_create", "sx_load_grid", "sx_add_source", "sx_step", "sx_sync",
              "sx_read_neutral_fraction", "sx_read_photons", "sx_destroy", "sx_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_0912_4273_gb300 import simplex as S

    bound = {name for name, _, _ in S._SIGS}
    assert set(_declared()) <= bound
    for n in _declared():
        assert hasattr(S, n)


def test_binding_constants_match_the_header():
    from paper_0912_4273_gb300 import simplex as S

    txt = open(os.path.join(ROOT, "include", "simplexgb.h")).read()
    defs = dict(re.findall(r"^#define\s+(SX_[A-Z_0-9]+)\s+(-?\d+)\b", txt, flags=re.M))
    assert "SX_STEP_BLOCK" in defs and "SX_MAX_BINS" in defs
    for name, val in defs.items():
        if hasattr(S, name):
            assert getattr(S, name) == int(val), name


def test_argument_errors_without_gpu(libpath):
    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    cfg = S.sx_config_default()
    assert cfg.nbins == 42 and cfg.precision == S.SX_FP32_TRANSPORT
    with pytest.raises(S.SimplexError) as e:
        S.sx_create(cfg, np.zeros((42, 3)))
    assert e.value.code == S.SX_EINVAL
    cfg.nbins = 0
    with pytest.raises((S.SimplexError, ValueError)):
        S.sx_create(cfg, np.zeros((0, 3)))
    cfg = S.sx_config_default()
    cfg.chem_frac = 1.5
    with pytest.raises(S.SimplexError) as e:
        S.sx_create(cfg, I.fibonacci_bins(42))
    assert e.value.code == S.SX_EINVAL
    cfg = S.sx_config_default()
    assert cfg.transport == S.SX_TRANSPORT_DCT and cfg.tau_switch == 1.0
    cfg.transport = 7
    with pytest.raises(S.SimplexError) as e:
        S.sx_create(cfg, I.fibonacci_bins(42))
    assert e.value.code == S.SX_EINVAL and "transport" in str(e.value)
    cfg = S.sx_config_default()
    cfg.transport = S.SX_TRANSPORT_COMBINED
    cfg.tau_switch = float("nan")
    with pytest.raises(S.SimplexError) as e:
        S.sx_create(cfg, I.fibonacci_bins(42))
    assert e.value.code == S.SX_EINVAL


def test_variant_and_autotune_argument_errors(libpath):
    """The launch-variant, autotune and budget-stepping calls reject a missing
    context before touching a GPU."""
    from paper_0912_4273_gb300 import simplex as S

    L = S.lib()
    assert L.sx_set_variant(None, 4) == S.SX_EINVAL
    v = ctypes.c_int32()
    assert L.sx_get_variant(None, ctypes.byref(v)) == S.SX_EINVAL
    r = S.sx_tune_result()
    assert L.sx_autotune(None, 1.0, 1, None, 0, ctypes.byref(r)) == S.SX_EINVAL
    assert L.sx_step_budgets(None, 1.0, 1, None) == S.SX_EINVAL


def test_checkpoint_argument_errors(libpath, tmp_path):
    """Checkpoint calls reject missing arguments and files that are not
    checkpoints without touching a GPU."""
    from paper_0912_4273_gb300 import simplex as S

    L = S.lib()
    assert L.sx_save(None, b"x") == S.SX_EINVAL
    assert L.sx_restore(None, b"x", None, 0) == S.SX_EINVAL
    n, nnz = ctypes.c_int64(), ctypes.c_int64()
    bad = tmp_path / "bad.sxck"
    bad.write_bytes(b"not a checkpoint")
    assert L.sx_checkpoint_info(str(bad).encode(), ctypes.byref(n), ctypes.byref(nnz)) == S.SX_EINVAL
    assert L.sx_checkpoint_info(str(tmp_path / "missing").encode(), ctypes.byref(n),
                                ctypes.byref(nnz)) == S.SX_EINVAL
    with pytest.raises(S.SimplexError):
        S.sx_checkpoint_info(str(bad))


def test_remesh_argument_errors(libpath):
    """sx_remesh_remove is host code: its refusals need no GPU."""
    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    L = S.lib()
    assert L.sx_remesh_remove(0, None, None, None, 0, None, None, 0, None, None) == S.SX_EINVAL
    p = I.stromgren_problem(500, seed=4)
    with pytest.raises(S.RemeshError) as e:  # an id out of range
        S.sx_remesh_remove(p.pos, p.row_ptr, p.col, p.simplices, p.volume, [p.n])
    assert e.value.code == S.SX_EINVAL and e.value.vertex == -1
    v = int(np.flatnonzero(p.interior)[3])
    with pytest.raises(S.RemeshError) as e:  # two adjacent vertices
        S.sx_remesh_remove(p.pos, p.row_ptr, p.col, p.simplices, p.volume, [v, int(p.col[p.row_ptr[v]])])
    assert e.value.vertex == -1
    # a malformed graph or tetrahedron list is refused before it is indexed
    tets = p.simplices.copy()
    tets[7, 2] = p.n
    col = p.col.copy()
    col[11] = -1
    rp = p.row_ptr.copy()
    rp[4] = rp[5] + 1
    for args in ((p.pos, p.row_ptr, p.col, tets), (p.pos, p.row_ptr, col, p.simplices),
                 (p.pos, rp, p.col, p.simplices)):
        with pytest.raises(S.RemeshError) as e:
            S.sx_remesh_remove(*args, p.volume, [v])
        assert e.value.code == S.SX_EINVAL and e.value.vertex == -1
    r = S.sx_remesh_remove(p.pos, p.row_ptr, p.col, p.simplices, p.volume, [])
    assert np.array_equal(r["col"], p.col) and np.array_equal(r["old_of_new"], np.arange(p.n))


def test_remesh_arrays_own_the_library_memory(libpath):
    """sx_remesh_remove's arrays are numpy views of the memory the library
    allocated: any one of them keeps the whole result alive, and the result
    is freed (sx_remesh_free) when the last one is gone."""
    import gc
    import weakref

    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    p = I.stromgren_problem(500, seed=4)
    v = int(np.flatnonzero(p.interior)[3])
    ref = S.sx_remesh_remove(p.pos, p.row_ptr, p.col, p.simplices, p.volume, [v])
    ref = {k: np.array(a) for k, a in ref.items()}  # copies
    r = S.sx_remesh_remove(p.pos, p.row_ptr, p.col, p.simplices, p.volume, [v])
    b = r["tets"]
    while not hasattr(b, "_owner"):
        b = b.base
    owner = weakref.ref(b._owner)
    del b
    tets = r["tets"][5:9]  # a view of a view
    del r
    gc.collect()
    assert owner() is not None
    assert np.array_equal(tets, ref["tets"][5:9])
    del tets
    gc.collect()
    assert owner() is None


def test_noalloc_refuses_a_decreasing_row_ptr(libpath):
    """A row_ptr that decreases is refused on the host, before any device
    work: its rows would index col out of range."""
    from paper_0912_4273_gb300 import inputs as I
    from paper_0912_4273_gb300 import simplex as S

    p = I.stromgren_problem(300, seed=2)
    rp = p.row_ptr.copy()
    rp[7] = rp[9] + 5  # row 6 overshoots, row 7 decreases
    out = ctypes.c_double(0.0)
    bins = np.ascontiguousarray(I.fibonacci_bins(21))
    P = ctypes.POINTER
    rc = S.lib().sx_kappa_noalloc(p.n, p.pos.ctypes.data_as(P(ctypes.c_double)),
                                  rp.ctypes.data_as(P(ctypes.c_int64)),
                                  p.col.ctypes.data_as(P(ctypes.c_int32)),
                                  p.flags.ctypes.data_as(P(ctypes.c_uint8)), 21,
                                  bins.ctypes.data_as(P(ctypes.c_double)), 0, None, ctypes.byref(out))
    assert rc == S.SX_EINVAL and "decrease" in S.sx_kappa_noalloc_last_error()
