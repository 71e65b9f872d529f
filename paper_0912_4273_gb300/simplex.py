"""Python binding of libsimplexgb.so (the C ABI of include/simplexgb.h).

Argument marshalling only: every step of the transport path runs in the CUDA
library.  The functions named ``sx_*`` mirror the C entry points one to one
and raise :class:`SimplexError` on a non-zero return.  :class:`Solver` bundles
them with a device workspace taken from PyTorch's allocator.

There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SX_OK, SX_EINVAL, SX_ENOMEM, SX_ECUDA, SX_ESTATE, SX_ETIMEOUT = 0, -1, -2, -3, -4, -5
SX_FP64, SX_FP32_TRANSPORT = 0, 1
SX_TRANSPORT_DCT, SX_TRANSPORT_BALLISTIC, SX_TRANSPORT_COMBINED = 0, 1, 2
SX_MAX_BINS = 128
SX_MAX_DEGREE = 64
SX_FLAG_SINK = 1
SX_FLAG_GHOST = 2
SX_STEP_BLOCK = 16  # steps whose rotation tables one launch makes


class SimplexError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"simplexgb error {code}: {msg}")
        self.code = code


class sx_config(C.Structure):
    _fields_ = [("nbins", C.c_int32), ("precision", C.c_int32), ("seed", C.c_uint64),
                ("sigma", C.c_double), ("alpha_B", C.c_double), ("kappa", C.c_double),
                ("chem_frac", C.c_double), ("chem_tol", C.c_double),
                ("chem_max_sub", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p),
                ("transport", C.c_int32), ("tau_switch", C.c_double), ("chem_fp32", C.c_int32),
                ("alpha_A", C.c_double)]


class sx_budget(C.Structure):
    _fields_ = [("emitted", C.c_double), ("absorbed", C.c_double), ("escaped", C.c_double),
                ("in_flight", C.c_double)]

    def as_dict(self):
        return dict(emitted=self.emitted, absorbed=self.absorbed, escaped=self.escaped,
                    in_flight=self.in_flight)


SX_TUNE_MAX_CANDIDATES = 4


class sx_remesh_result(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("ntet", C.c_int64),
                ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
                ("volume", C.POINTER(C.c_double)), ("tets", C.POINTER(C.c_int32)),
                ("old_of_new", C.POINTER(C.c_int32)), ("bad_vertex", C.c_int32)]


class sx_tune_result(C.Structure):
    _fields_ = [("variant", C.c_int32), ("ncandidates", C.c_int32),
                ("candidates", C.c_int32 * SX_TUNE_MAX_CANDIDATES),
                ("ms_per_step", C.c_double * SX_TUNE_MAX_CANDIDATES),
                ("stride", C.c_int32), ("strides", C.c_int32 * SX_TUNE_MAX_CANDIDATES)]


class sx_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("step", C.c_int64),
                ("workspace_bytes", C.c_int64), ("kappa", C.c_double),
                ("subcycles", C.c_int64), ("capped", C.c_int64), ("max_degree", C.c_int32),
                ("nsources", C.c_int32), ("step_kernel_ms", C.c_double),
                ("step_kernel_launches", C.c_int64), ("index_errors", C.c_int64)]


_LIB = None
_LOCK = threading.Lock()

# (name, restype, argtypes) of every entry point of include/simplexgb.h
_P = C.POINTER
_SIGS = [
    ("sx_config_default", None, [_P(sx_config)]),
    ("sx_create", C.c_int, [_P(sx_config), _P(C.c_double), _P(C.c_void_p)]),
    ("sx_workspace_bytes", C.c_int, [C.c_void_p, C.c_int64, C.c_int64, _P(C.c_int64)]),
    ("sx_load_grid", C.c_int, [C.c_void_p, C.c_int64, _P(C.c_double), _P(C.c_int64),
                               _P(C.c_int32), _P(C.c_double), _P(C.c_double), _P(C.c_uint8),
                               _P(C.c_double), C.c_void_p, C.c_int64]),
    ("sx_add_source", C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
    ("sx_step", C.c_int, [C.c_void_p, C.c_double, C.c_int32]),
    ("sx_step_budgets", C.c_int, [C.c_void_p, C.c_double, C.c_int32, _P(sx_budget)]),
    ("sx_sync", C.c_int, [C.c_void_p]),
    ("sx_read_neutral_fraction", C.c_int, [C.c_void_p, _P(C.c_double)]),
    ("sx_read_photons", C.c_int, [C.c_void_p, _P(C.c_double), _P(sx_budget)]),
    ("sx_get_info", C.c_int, [C.c_void_p, _P(sx_info)]),
    ("sx_profile", C.c_int, [C.c_void_p, C.c_int]),
    ("sx_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("sx_checkpoint_info", C.c_int, [C.c_char_p, _P(C.c_int64), _P(C.c_int64)]),
    ("sx_restore", C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p, C.c_int64]),
    ("sx_checkpoint_verify", C.c_int, [C.c_char_p]),
    ("sx_set_variant", C.c_int, [C.c_void_p, C.c_int32]),
    ("sx_get_variant", C.c_int, [C.c_void_p, _P(C.c_int32)]),
    ("sx_set_bin_stride", C.c_int, [C.c_void_p, C.c_int32]),
    ("sx_get_bin_stride", C.c_int, [C.c_void_p, _P(C.c_int32)]),
    ("sx_autotune", C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_size_t,
                              _P(sx_tune_result)]),
    ("sx_grid_update_mark", C.c_int, [C.c_void_p, C.c_double, C.c_double, _P(C.c_int32),
                                      _P(C.c_int64)]),
    ("sx_grid_update_apply", C.c_int, [C.c_void_p, C.c_int64, _P(C.c_double), _P(C.c_int64),
                                       _P(C.c_int32), _P(C.c_double), _P(C.c_double),
                                       _P(C.c_uint8), _P(C.c_int32), C.c_void_p, C.c_int64]),
    ("sx_destroy", None, [C.c_void_p]),
    ("sx_last_error", C.c_char_p, [C.c_void_p]),
    ("sx_batch_workspace_bytes", C.c_int, [C.c_int32, _P(C.c_int64)]),
    ("sx_batch_create", C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64,
                                  _P(C.c_void_p)]),
    ("sx_batch_step", C.c_int, [C.c_void_p, _P(C.c_void_p), C.c_int32, _P(C.c_double),
                                C.c_int32]),
    ("sx_batch_destroy", None, [C.c_void_p]),
    ("sx_batch_last_error", C.c_char_p, [C.c_void_p]),
    ("sx_kappa_noalloc", C.c_int, [C.c_int64, _P(C.c_double), _P(C.c_int64), _P(C.c_int32),
                                   _P(C.c_uint8), C.c_int32, _P(C.c_double), C.c_int32,
                                   C.c_void_p, _P(C.c_double)]),
    ("sx_kappa_noalloc_last_error", C.c_char_p, []),
    ("sx_remesh_remove", C.c_int, [C.c_int64, _P(C.c_double), _P(C.c_int64), _P(C.c_int32),
                                   C.c_int64, _P(C.c_int32), _P(C.c_double), C.c_int64,
                                   _P(C.c_int32), _P(sx_remesh_result)]),
    ("sx_remesh_free", None, [_P(sx_remesh_result)]),
    ("sx_kappa_sums", C.c_int, [C.c_void_p, _P(C.c_double), _P(C.c_double)]),
    ("sx_halo_bytes", C.c_int, [C.c_void_p, C.c_int64, C.c_int64, _P(C.c_int64)]),
    ("sx_set_photon_unit", C.c_int, [C.c_void_p, C.c_double]),
    ("sx_halo_pack", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                               C.c_void_p]),
    ("sx_halo_unpack", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_void_p]),
]


def library_path() -> str:
    """The in-tree build, unless $SIMPLEXGB_LIBRARY names another build of it."""
    return os.environ.get("SIMPLEXGB_LIBRARY") or _build.lib_path()


def lib():
    """Load libsimplexgb.so (built in-tree by ``build()``); raise if it is missing."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is not built; run __graft_entry__.build() first")
            L = C.CDLL(path)
            for name, res, args in _SIGS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _check(ctx, rc: int):
    if rc != SX_OK:
        msg = lib().sx_last_error(ctx)
        raise SimplexError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# One-to-one wrappers of the C entry points
# ---------------------------------------------------------------------------
def sx_config_default() -> sx_config:
    cfg = sx_config()
    lib().sx_config_default(C.byref(cfg))
    return cfg


def sx_create(cfg: sx_config, bin_dirs):
    """bin_dirs: nbins x 3 unit vectors, or None for the library's Fibonacci
    lattice."""
    ctx = C.c_void_p()
    if bin_dirs is None:
        _check(None, lib().sx_create(C.byref(cfg), None, C.byref(ctx)))
        return ctx
    b = np.ascontiguousarray(bin_dirs, dtype=np.float64)
    if b.shape != (cfg.nbins, 3):
        raise ValueError("bin_dirs must be nbins x 3")
    _check(None, lib().sx_create(C.byref(cfg), _ptr(b, C.c_double), C.byref(ctx)))
    return ctx


def sx_workspace_bytes(ctx, n: int, nnz: int) -> int:
    out = C.c_int64()
    _check(ctx, lib().sx_workspace_bytes(ctx, n, nnz, C.byref(out)))
    return out.value


def sx_load_grid(ctx, n, pos, row_ptr, col, nH, volume, flags, y0, d_workspace: int,
                 workspace_bytes: int):
    y0p = None if y0 is None else _ptr(y0, C.c_double)
    _check(ctx, lib().sx_load_grid(ctx, n, _ptr(pos, C.c_double), _ptr(row_ptr, C.c_int64),
                                   _ptr(col, C.c_int32), _ptr(nH, C.c_double),
                                   _ptr(volume, C.c_double), _ptr(flags, C.c_uint8), y0p,
                                   C.c_void_p(d_workspace), workspace_bytes))


def sx_add_source(ctx, vertex: int, photons_per_s: float):
    _check(ctx, lib().sx_add_source(ctx, int(vertex), float(photons_per_s)))


def sx_step(ctx, dt_s: float, nsteps: int):
    _check(ctx, lib().sx_step(ctx, float(dt_s), int(nsteps)))


def sx_step_budgets(ctx, dt_s: float, nsteps: int, budgets: np.ndarray):
    """budgets: float64 array of nsteps x 4 (emitted, absorbed, escaped, in
    flight), filled once the stream has reached the steps (sx_sync)."""
    if budgets.dtype != np.float64 or budgets.shape != (nsteps, 4) or not budgets.flags.c_contiguous:
        raise ValueError("budgets must be a C-contiguous float64 array of nsteps x 4")
    _check(ctx, lib().sx_step_budgets(ctx, float(dt_s), int(nsteps),
                                      budgets.ctypes.data_as(C.POINTER(sx_budget))))


class RemeshError(ValueError):
    """A cavity could not be re-triangulated locally (``vertex`` is the
    removed vertex), or the removal is invalid (``vertex`` is -1)."""

    def __init__(self, code: int, vertex: int):
        super().__init__(f"sx_remesh_remove: code {code}, vertex {vertex}")
        self.code = code
        self.vertex = vertex


def sx_remesh_free(result: "sx_remesh_result"):
    """Free the arrays of a result of the C call sx_remesh_remove."""
    lib().sx_remesh_free(C.byref(result))


class _RemeshArrays:
    """Owns the arrays of one sx_remesh_remove result and frees them when the
    last numpy array over any of them is gone."""

    def __init__(self, res: "sx_remesh_result"):
        self.res = res
        self._free = lib().sx_remesh_free  # bound now: no lock in the finaliser

    def view(self, ptr, ctype, count: int, dtype, shape=None) -> np.ndarray:
        if count == 0:
            a = np.empty(0, dtype=dtype)
        else:
            buf = (ctype * count).from_address(C.cast(ptr, C.c_void_p).value)
            buf._owner = self  # every array over the result keeps it alive
            a = np.frombuffer(buf, dtype=dtype)
        return a.reshape(shape) if shape is not None else a

    def __del__(self):
        try:
            self._free(C.byref(self.res))
        except Exception:
            pass


def sx_remesh_remove(pos, row_ptr, col, tets, volume, removed) -> dict:
    """The grid without the `removed` vertices (see include/simplexgb.h):
    dict of row_ptr, col, volume, tets, old_of_new.  The arrays lie in the
    memory the library allocated (no copy); it is freed when the last of
    them is gone."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    tt = np.ascontiguousarray(tets, dtype=np.int32)
    vol = np.ascontiguousarray(volume, dtype=np.float64)
    rem = np.ascontiguousarray(removed, dtype=np.int32)
    res = sx_remesh_result()
    rc = lib().sx_remesh_remove(len(pos), _ptr(pos, C.c_double), _ptr(rp, C.c_int64),
                                _ptr(cl, C.c_int32), len(tt), _ptr(tt, C.c_int32),
                                _ptr(vol, C.c_double), len(rem), _ptr(rem, C.c_int32), C.byref(res))
    if rc != SX_OK:
        raise RemeshError(rc, res.bad_vertex)
    owner = _RemeshArrays(res)
    return dict(row_ptr=owner.view(res.row_ptr, C.c_int64, res.n + 1, np.int64),
                col=owner.view(res.col, C.c_int32, res.nnz, np.int32),
                volume=owner.view(res.volume, C.c_double, res.n, np.float64),
                tets=owner.view(res.tets, C.c_int32, 4 * res.ntet, np.int32, (res.ntet, 4)),
                old_of_new=owner.view(res.old_of_new, C.c_int32, res.n, np.int32))


def sx_sync(ctx):
    _check(ctx, lib().sx_sync(ctx))


def sx_read_neutral_fraction(ctx, out: np.ndarray):
    _check(ctx, lib().sx_read_neutral_fraction(ctx, _ptr(out, C.c_double)))


def sx_read_photons(ctx, per_vertex=None) -> sx_budget:
    b = sx_budget()
    pv = None if per_vertex is None else _ptr(per_vertex, C.c_double)
    _check(ctx, lib().sx_read_photons(ctx, pv, C.byref(b)))
    return b


def sx_get_info(ctx) -> sx_info:
    info = sx_info()
    _check(ctx, lib().sx_get_info(ctx, C.byref(info)))
    return info


def sx_profile(ctx, enable: bool):
    _check(ctx, lib().sx_profile(ctx, 1 if enable else 0))


def sx_save(ctx, path: str):
    _check(ctx, lib().sx_save(ctx, os.fsencode(path)))


def sx_checkpoint_info(path: str):
    n, nnz = C.c_int64(), C.c_int64()
    rc = lib().sx_checkpoint_info(os.fsencode(path), C.byref(n), C.byref(nnz))
    if rc != SX_OK:
        raise SimplexError(rc, f"{path} is not a checkpoint")
    return n.value, nnz.value


def sx_checkpoint_verify(path: str):
    """Check a checkpoint file against its checksum (no GPU); raises
    SimplexError with the reason if it is not an intact checkpoint."""
    rc = lib().sx_checkpoint_verify(os.fsencode(path))
    if rc != SX_OK:
        raise SimplexError(rc, sx_last_error(None))


def sx_restore(ctx, path: str, ws_ptr: int, ws_bytes: int):
    _check(ctx, lib().sx_restore(ctx, os.fsencode(path), C.c_void_p(ws_ptr), ws_bytes))


def sx_set_variant(ctx, variant: int):
    _check(ctx, lib().sx_set_variant(ctx, variant))


def sx_get_variant(ctx) -> int:
    v = C.c_int32()
    _check(ctx, lib().sx_get_variant(ctx, C.byref(v)))
    return v.value


def sx_set_bin_stride(ctx, stride: int):
    _check(ctx, lib().sx_set_bin_stride(ctx, stride))


def sx_get_bin_stride(ctx) -> int:
    v = C.c_int32()
    _check(ctx, lib().sx_get_bin_stride(ctx, C.byref(v)))
    return v.value


def sx_autotune(ctx, dt: float, nsteps: int, scratch_ptr: int, scratch_bytes: int) -> sx_tune_result:
    r = sx_tune_result()
    _check(ctx, lib().sx_autotune(ctx, dt, nsteps, C.c_void_p(scratch_ptr), scratch_bytes,
                                  C.byref(r)))
    return r


def sx_grid_update_mark(ctx, y_thresh: float, min_spacing: float, n: int) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.int32)
    k = C.c_int64()
    _check(ctx, lib().sx_grid_update_mark(ctx, y_thresh, min_spacing, _ptr(out, C.c_int32),
                                          C.byref(k)))
    return out[:k.value].copy()


def sx_grid_update_apply(ctx, n_new, pos, row_ptr, col, nH, volume, flags, old_of_new,
                         d_workspace: int, workspace_bytes: int):
    _check(ctx, lib().sx_grid_update_apply(ctx, n_new, _ptr(pos, C.c_double),
                                           _ptr(row_ptr, C.c_int64), _ptr(col, C.c_int32),
                                           _ptr(nH, C.c_double), _ptr(volume, C.c_double),
                                           _ptr(flags, C.c_uint8), _ptr(old_of_new, C.c_int32),
                                           C.c_void_p(d_workspace), workspace_bytes))


def sx_kappa_sums(ctx):
    """(num, den) of kappa over the loaded grid's interior, non-ghost vertices."""
    a, b = C.c_double(), C.c_double()
    _check(ctx, lib().sx_kappa_sums(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def sx_set_photon_unit(ctx, unit: float):
    _check(ctx, lib().sx_set_photon_unit(ctx, float(unit)))


def sx_halo_bytes(ctx, n_edges: int, n_rows: int) -> int:
    out = C.c_int64()
    _check(ctx, lib().sx_halo_bytes(ctx, n_edges, n_rows, C.byref(out)))
    return out.value


def sx_halo_pack(ctx, n_edges: int, d_edge_idx: int, n_rows: int, d_row_idx: int, d_buf: int):
    """Device pointers (ints): int32 in-edge and vertex indices, the buffer."""
    _check(ctx, lib().sx_halo_pack(ctx, n_edges, C.c_void_p(d_edge_idx), n_rows,
                                   C.c_void_p(d_row_idx), C.c_void_p(d_buf)))


def sx_halo_unpack(ctx, n_edges: int, d_edge_idx: int, n_rows: int, d_row_idx: int, d_buf: int):
    _check(ctx, lib().sx_halo_unpack(ctx, n_edges, C.c_void_p(d_edge_idx), n_rows,
                                     C.c_void_p(d_row_idx), C.c_void_p(d_buf)))


def sx_destroy(ctx):
    lib().sx_destroy(ctx)


def sx_last_error(ctx=None) -> str:
    m = lib().sx_last_error(ctx)
    return m.decode() if m else ""


def _bcheck(batch, rc: int):
    if rc != SX_OK:
        msg = lib().sx_batch_last_error(batch)
        raise SimplexError(rc, msg.decode() if msg else "")


def sx_batch_workspace_bytes(max_grids: int) -> int:
    out = C.c_int64()
    _bcheck(None, lib().sx_batch_workspace_bytes(max_grids, C.byref(out)))
    return out.value


def sx_batch_create(max_grids: int, device: int, stream: int, d_workspace: int,
                    workspace_bytes: int):
    out = C.c_void_p()
    _bcheck(None, lib().sx_batch_create(max_grids, device, C.c_void_p(stream),
                                        C.c_void_p(d_workspace), workspace_bytes, C.byref(out)))
    return out


def sx_batch_step(batch, ctxs, dts, nsteps: int):
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    d = np.ascontiguousarray(dts, dtype=np.float64)
    _bcheck(batch, lib().sx_batch_step(batch, arr, n, _ptr(d, C.c_double), nsteps))


def sx_batch_destroy(batch):
    lib().sx_batch_destroy(batch)


def sx_batch_last_error(batch=None) -> str:
    m = lib().sx_batch_last_error(batch)
    return m.decode() if m else ""


SX_NOALLOC_MAX_VERTICES = 16384
SX_NOALLOC_MAX_EDGES = 262144


def sx_kappa_noalloc(n, pos, row_ptr, col, flags, bin_dirs, device: int = 0, stream: int = 0) -> float:
    """kappa of a grid without any device allocation (see include/simplexgb.h)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    b = np.ascontiguousarray(bin_dirs, dtype=np.float64)
    out = C.c_double()
    rc = lib().sx_kappa_noalloc(n, _ptr(pos, C.c_double), _ptr(rp, C.c_int64), _ptr(cl, C.c_int32),
                                _ptr(fl, C.c_uint8), len(b), _ptr(b, C.c_double), device,
                                C.c_void_p(stream), C.byref(out))
    if rc != SX_OK:
        raise SimplexError(rc, sx_kappa_noalloc_last_error())
    return out.value


def sx_kappa_noalloc_last_error() -> str:
    m = lib().sx_kappa_noalloc_last_error()
    return m.decode() if m else ""


class Batch:
    """Steps many :class:`Solver` grids together (one persistent launch per step)."""

    def __init__(self, max_grids: int, device: int = 0, stream=None):
        import torch

        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = sx_batch_workspace_bytes(max_grids)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.workspace.record_stream(self.stream)  # freed memory waits for this stream's work
        self.handle = sx_batch_create(max_grids, device, self.stream.cuda_stream,
                                      self.workspace.data_ptr(), nbytes)

    def step(self, solvers, dts, nsteps: int = 1):
        if np.isscalar(dts):
            dts = [dts] * len(solvers)
        sx_batch_step(self.handle, [s.ctx for s in solvers], dts, nsteps)

    def close(self):
        if getattr(self, "handle", None):
            sx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Convenience: one grid with a torch-allocated device workspace
# ---------------------------------------------------------------------------
class Solver:
    """A SimpleX2 solve of one grid on one GPU: direction-conserving (default),
    ballistic or combined transport (``transport``, ``tau_switch``).

    The workspace (per-grid device state) is a torch uint8 tensor on the
    context's device, so that memory comes from PyTorch's caching allocator;
    ``stream`` is a ``torch.cuda.Stream`` (default: the current stream).
    Every workspace is marked as used on that stream, so the allocator does
    not hand its memory out again (after ``close``, a reload or an update)
    before the steps queued there have run.
    """

    def __init__(self, bins: np.ndarray, precision: int = SX_FP32_TRANSPORT, seed: int = 0,
                 device: int = 0, stream=None, sigma: float = 6.3e-18, alpha_B: float = 2.59e-13,
                 kappa: float = 0.0, chem_frac: float = 0.5, chem_tol: float = 1e-5,
                 chem_max_sub: int = 1000, transport: int = SX_TRANSPORT_DCT,
                 tau_switch: float = 1.0, chem_fp32: bool = False, alpha_A: float = 0.0):
        import torch

        self._torch = torch
        # an integer: that many bins on the library's Fibonacci lattice
        nbins = int(bins) if np.isscalar(bins) else len(bins)
        cfg = sx_config_default()
        cfg.nbins = nbins
        cfg.precision = precision
        cfg.seed = seed
        cfg.sigma = sigma
        cfg.alpha_B = alpha_B
        cfg.kappa = kappa
        cfg.chem_frac = chem_frac
        cfg.chem_tol = chem_tol
        cfg.chem_max_sub = chem_max_sub
        cfg.transport = transport
        cfg.tau_switch = tau_switch
        cfg.chem_fp32 = 1 if chem_fp32 else 0
        cfg.alpha_A = alpha_A
        cfg.device = device
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfg.stream = C.c_void_p(self.stream.cuda_stream)
        self.cfg = cfg
        self.nbins = nbins
        self.ctx = sx_create(cfg, None if np.isscalar(bins) else bins)
        self.workspace = None
        self.n = 0

    def workspace_bytes(self, n: int, nnz: int) -> int:
        return sx_workspace_bytes(self.ctx, n, nnz)

    def _new_workspace(self, nbytes: int):
        ws = self._torch.empty(nbytes, dtype=self._torch.uint8, device=self.device)
        ws.record_stream(self.stream)
        return ws

    def load(self, problem=None, *, pos=None, row_ptr=None, col=None, nH=None, volume=None,
             flags=None, y0=None, workspace=None):
        if problem is not None:
            pos, row_ptr, col = problem.pos, problem.row_ptr, problem.col
            nH, volume, flags = problem.nH, problem.volume, problem.flags
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        nH = np.ascontiguousarray(nH, dtype=np.float64)
        volume = np.ascontiguousarray(volume, dtype=np.float64)
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
        n = len(pos)
        nbytes = self.workspace_bytes(n, int(row_ptr[-1]))
        if workspace is None:
            workspace = self._new_workspace(nbytes)
        else:
            workspace.record_stream(self.stream)
        self.workspace = workspace
        sx_load_grid(self.ctx, n, pos, row_ptr, col, nH, volume, flags, y0,
                     workspace.data_ptr(), workspace.numel())
        self.n = n
        if problem is not None:
            for v, r in zip(problem.src_vertex, problem.src_rate):
                self.add_source(int(v), float(r))
        return self

    def add_source(self, vertex: int, photons_per_s: float):
        sx_add_source(self.ctx, vertex, photons_per_s)

    def step(self, dt: float, nsteps: int = 1):
        sx_step(self.ctx, dt, nsteps)

    def step_budgets(self, dt: float, nsteps: int, out: np.ndarray = None) -> np.ndarray:
        """Steps, each followed by a queued read of the photon budget into row
        k of `out` (nsteps x 4 float64: emitted, absorbed, escaped, in
        flight; page-locked memory keeps the copies asynchronous).  The rows
        are filled once the stream reaches them (``sync``)."""
        if out is None:
            out = np.empty((nsteps, 4), dtype=np.float64)
        sx_step_budgets(self.ctx, dt, nsteps, out)
        return out

    def sync(self):
        sx_sync(self.ctx)

    @property
    def y(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        sx_read_neutral_fraction(self.ctx, out)
        return out

    @property
    def budget(self) -> dict:
        return sx_read_photons(self.ctx).as_dict()

    def photons(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        sx_read_photons(self.ctx, out)
        return out

    def mark_removal(self, y_thresh: float, min_spacing: float) -> np.ndarray:
        """Vertices the dynamic grid update would remove (ascending ids)."""
        return sx_grid_update_mark(self.ctx, y_thresh, min_spacing, self.n)

    def apply_update(self, problem_new, old_of_new):
        """Continue on the re-triangulated survivors (state carried over)."""
        pos = np.ascontiguousarray(problem_new.pos, dtype=np.float64)
        rp = np.ascontiguousarray(problem_new.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(problem_new.col, dtype=np.int32)
        nH = np.ascontiguousarray(problem_new.nH, dtype=np.float64)
        vol = np.ascontiguousarray(problem_new.volume, dtype=np.float64)
        fl = np.ascontiguousarray(problem_new.flags, dtype=np.uint8)
        o2n = np.ascontiguousarray(old_of_new, dtype=np.int32)
        ws = self._new_workspace(self.workspace_bytes(len(pos), int(rp[-1])))
        sx_grid_update_apply(self.ctx, len(pos), pos, rp, col, nH, vol, fl, o2n, ws.data_ptr(),
                             ws.numel())
        self.workspace = ws
        self.n = len(pos)
        return self

    def profile(self, enable: bool = True):
        sx_profile(self.ctx, enable)

    def save(self, path: str):
        """Write the grid and its state to a checkpoint file."""
        sx_save(self.ctx, path)

    def restore(self, path: str):
        """Replace the grid and state by a checkpoint's (same bins and
        precision); the workspace is allocated here for its size."""
        n, nnz = sx_checkpoint_info(path)
        ws = self._new_workspace(self.workspace_bytes(n, nnz))
        sx_restore(self.ctx, path, ws.data_ptr(), ws.numel())
        self.workspace = ws
        self.n = n
        return self

    @property
    def variant(self) -> int:
        """Vertices per warp of the step kernel (2 or 4)."""
        return sx_get_variant(self.ctx)

    @variant.setter
    def variant(self, v: int):
        sx_set_variant(self.ctx, int(v))

    def autotune(self, dt: float, nsteps: int = 4) -> dict:
        """Time every step-kernel variant for nsteps steps from the current
        state and keep the fastest; the state is saved in a scratch copy of
        the workspace (allocated here for the call) and restored."""
        scratch = self._new_workspace(self.workspace.numel())
        try:
            r = sx_autotune(self.ctx, dt, nsteps, scratch.data_ptr(), scratch.numel())
        finally:
            del scratch
        k = r.ncandidates
        return dict(variant=r.variant, stride=r.stride, candidates=list(r.candidates[:k]),
                    strides=list(r.strides[:k]), ms_per_step=list(r.ms_per_step[:k]))

    @property
    def bin_stride(self) -> int:
        """Row stride of the stored photons (nbins rounded up to 4 or 8)."""
        return sx_get_bin_stride(self.ctx)

    @bin_stride.setter
    def bin_stride(self, v: int):
        sx_set_bin_stride(self.ctx, int(v))

    @property
    def info(self) -> dict:
        i = sx_get_info(self.ctx)
        return {k: getattr(i, k) for k, _ in sx_info._fields_}

    def close(self):
        if getattr(self, "ctx", None):
            sx_destroy(self.ctx)
            self.ctx = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
