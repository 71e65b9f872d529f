"""ctypes front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

What lives here:
  * ``build()`` -- compiles ``sx_oracle.c`` and ``delaunay3d.c`` with gcc;
  * thin wrappers of the C entry points (Philox, rotation, tables, chemistry,
    the DCT sweep with optional diffuse recombination radiation, the
    Delaunay builder);
  * the analytic Test-1 solutions of Sect. 5.1: Stromgren radius
    (Eq. stromgren_radius), I-front history (Eq. IFront_pos, IFront_vel) and
    the equilibrium ionisation profile (Eq. inner_stromgren_region).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRCS = ["sx_oracle.c", "delaunay3d.c"]
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle.so")
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    # OpenMP for the threaded sweep (OracleSim(threads=...)); without it the
    # same code runs on one thread
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            d, i64, i32, u8 = C.c_double, C.c_int64, C.c_int32, C.c_uint8
            P = C.POINTER
            L.ox_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.ox_rotation.argtypes = [C.c_uint64, i64, P(d)]
            L.ox_rotation.restype = C.c_int
            L.ox_rotated_bins.argtypes = [P(d), C.c_int, P(d), P(i32)]
            L.ox_bin_map.argtypes = [C.c_int, P(i32), P(i32), P(i32)]
            L.ox_edge_tables.argtypes = [i64, P(d), P(i64), P(i32), P(i32), P(u8), P(d)]
            L.ox_kappa.argtypes = [i64, P(d), P(i64), P(i32), P(u8), P(i32), P(u8), C.c_int, P(d)]
            L.ox_kappa.restype = d
            L.ox_chem.argtypes = [P(d), d, d, d, d, d, d, d, C.c_int, P(C.c_int), P(C.c_int)]
            L.ox_chem.restype = d
            L.ox_chem_rec.argtypes = [P(d), d, d, d, d, d, d, d, C.c_int, P(C.c_int), P(C.c_int), P(d)]
            L.ox_chem_rec.restype = d
            L.ox_get_diffuse.argtypes = [C.c_void_p, P(d)]
            L.ox_get_diffuse.restype = d
            L.ox_create.argtypes = [C.c_void_p, i64, P(d), P(i64), P(i32), P(d), P(d), P(u8), P(d),
                                    P(d)]
            L.ox_create.restype = C.c_void_p
            L.ox_destroy.argtypes = [C.c_void_p]
            L.ox_add_source.argtypes = [C.c_void_p, i32, d]
            L.ox_add_source.restype = C.c_int
            L.ox_step.argtypes = [C.c_void_p, d, C.c_int]
            L.ox_set_threads.argtypes = [C.c_void_p, C.c_int]
            for name in ("ox_get_y", "ox_set_y", "ox_get_I", "ox_set_I", "ox_get_budget"):
                getattr(L, name).argtypes = [C.c_void_p, P(d)]
            L.ox_get_kappa.argtypes = [C.c_void_p]
            L.ox_get_kappa.restype = d
            L.ox_get_step.argtypes = [C.c_void_p]
            L.ox_get_step.restype = i64
            L.ox_get_stats.argtypes = [C.c_void_p, P(i64)]
            L.ox_get_vertex_consts.argtypes = [C.c_void_p, P(d), P(d), P(d)]
            L.ox_get_tables.argtypes = [C.c_void_p, P(i32), P(u8), P(d)]
            L.ox_associate_all.argtypes = [C.c_void_p, i64, P(i32)]
            L.ox_mark_removal.argtypes = [C.c_void_p, d, d, P(i32)]
            L.ox_mark_removal.restype = i64
            L.ox_hand_over.argtypes = [C.c_void_p, i64, P(i32), P(d)]
            L.ox_set_step.argtypes = [C.c_void_p, i64]
            L.ox_get_inflight.argtypes = [C.c_void_p, P(d)]
            L.ox_get_ballistic.argtypes = [C.c_void_p, P(u8), P(i64), P(u8)]
            L.ox_set_budget.argtypes = [C.c_void_p, P(d)]
            L.dl_triangulate.argtypes = [i64, P(d), P(P(i32))]
            L.dl_triangulate.restype = i64
            L.dl_free.argtypes = [P(i32)]
            L.dl_insphere.argtypes = [P(d)] * 5
            L.dl_insphere.restype = C.c_int
            _LIB = L
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---------------------------------------------------------------------------
# Pieces
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().ox_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def rotation(seed: int, step: int):
    R = np.zeros(9, dtype=np.float64)
    att = lib().ox_rotation(C.c_uint64(seed), step, _p(R, C.c_double))
    return R.reshape(3, 3), att


def rotated_bins(R, bins) -> np.ndarray:
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(9))
    b = np.ascontiguousarray(bins, dtype=np.float64)
    q = np.zeros((len(b), 3), dtype=np.int32)
    lib().ox_rotated_bins(_p(R, C.c_double), len(b), _p(b, C.c_double), _p(q, C.c_int32))
    return q


def bin_map(q_old, q_new) -> np.ndarray:
    """Closest new bin of every old bin (exact integer dots, ties -> lowest)."""
    a = np.ascontiguousarray(q_old, dtype=np.int32)
    b = np.ascontiguousarray(q_new, dtype=np.int32)
    out = np.zeros(len(a), dtype=np.int32)
    lib().ox_bin_map(len(a), _p(a, C.c_int32), _p(b, C.c_int32), _p(out, C.c_int32))
    return out


def edge_tables(pos, row_ptr, col):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n, nnz = len(pos), int(rp[-1])
    q = np.zeros((max(nnz, 1), 3), dtype=np.int32)
    st = np.zeros((max(nnz, 1), 4), dtype=np.uint8)
    ml = np.zeros(n, dtype=np.float64)
    lib().ox_edge_tables(n, _p(pos, C.c_double), _p(rp, C.c_int64), _p(cl, C.c_int32),
                         _p(q, C.c_int32), _p(st, C.c_uint8), _p(ml, C.c_double))
    return q[:nnz], st[:nnz], ml


def chem(y: float, N_in: float, dt: float, A: float, tau_max: float, R0: float,
         fc: float = 0.5, tol: float = 1e-5, max_sub: int = 1000):
    """One cell over one step; returns (y_new, transmitted fraction, nsub, capped)."""
    yy = C.c_double(y)
    ns = C.c_int(0)
    cp = C.c_int(0)
    f = lib().ox_chem(C.byref(yy), N_in, dt, A, tau_max, R0, fc, tol, max_sub, C.byref(ns),
                      C.byref(cp))
    return yy.value, f, ns.value, cp.value


def chem_rec(y: float, N_in: float, dt: float, A: float, tau_max: float, R0: float,
             fc: float = 0.5, tol: float = 1e-5, max_sub: int = 1000):
    """As ``chem``, and the recombinations per atom during the step:
    returns (y_new, transmitted fraction, recombinations per atom, nsub, capped)."""
    yy = C.c_double(y)
    ns = C.c_int(0)
    cp = C.c_int(0)
    rec = C.c_double(0.0)
    f = lib().ox_chem_rec(C.byref(yy), N_in, dt, A, tau_max, R0, fc, tol, max_sub, C.byref(ns),
                          C.byref(cp), C.byref(rec))
    return yy.value, f, rec.value, ns.value, cp.value


# ---------------------------------------------------------------------------
# The sweep
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    nbins: int = 42
    seed: int = 0
    sigma: float = 6.3e-18
    alpha_B: float = 2.59e-13
    kappa: float = 0.0          # <= 0: compute from the grid
    chem_frac: float = 0.5
    chem_tol: float = 1e-5
    chem_max_sub: int = 1000
    transport: int = 0          # 0 direction conserving, 1 ballistic, 2 combined
    tau_switch: float = 1.0     # combined: ballistic where y tau_max >= tau_switch (Sect. 5.1.3)
    alpha_A: float = 0.0        # 0: on-the-spot (case B); > 0: case A with the ground-level
                                # recombination photons re-emitted (Sect. 2.2.1)


class _CParams(C.Structure):
    _fields_ = [("nbins", C.c_int), ("seed", C.c_uint64), ("sigma", C.c_double),
                ("alpha_B", C.c_double), ("kappa", C.c_double), ("chem_frac", C.c_double),
                ("chem_tol", C.c_double), ("chem_max_sub", C.c_int), ("transport", C.c_int),
                ("tau_switch", C.c_double), ("alpha_A", C.c_double)]


class OracleSim:
    """FP64 SimpleX2 simulation of one grid on the CPU: direction-conserving,
    ballistic or combined transport (``Params.transport``)."""

    def __init__(self, problem, params: Params, bins: np.ndarray, y0=None, threads: int = 1):
        """threads > 1: the direction-conserving sweep runs on that many
        threads, with the serial sweep's results bit for bit."""
        L = lib()
        self.p = params
        self.n = problem.n
        self.nbins = params.nbins
        self._keep = dict(
            pos=np.ascontiguousarray(problem.pos, dtype=np.float64),
            rp=np.ascontiguousarray(problem.row_ptr, dtype=np.int64),
            col=np.ascontiguousarray(problem.col, dtype=np.int32),
            nH=np.ascontiguousarray(problem.nH, dtype=np.float64),
            vol=np.ascontiguousarray(problem.volume, dtype=np.float64),
            flags=np.ascontiguousarray(problem.flags, dtype=np.uint8),
            bins=np.ascontiguousarray(bins, dtype=np.float64),
        )
        assert self._keep["bins"].shape == (params.nbins, 3)
        k = self._keep
        cp = _CParams(params.nbins, params.seed, params.sigma, params.alpha_B, params.kappa,
                      params.chem_frac, params.chem_tol, params.chem_max_sub, params.transport,
                      params.tau_switch, params.alpha_A)
        y0p = None
        if y0 is not None:
            k["y0"] = np.ascontiguousarray(y0, dtype=np.float64)
            y0p = _p(k["y0"], C.c_double)
        self.h = L.ox_create(C.byref(cp), self.n, _p(k["pos"], C.c_double), _p(k["rp"], C.c_int64),
                             _p(k["col"], C.c_int32), _p(k["nH"], C.c_double),
                             _p(k["vol"], C.c_double), _p(k["flags"], C.c_uint8), y0p,
                             _p(k["bins"], C.c_double))
        if not self.h:
            raise ValueError("diffuse radiation needs alpha_A >= alpha_B")
        L.ox_set_threads(self.h, int(threads))
        for v, r in zip(problem.src_vertex, problem.src_rate):
            if L.ox_add_source(self.h, int(v), float(r)) != 0:
                raise ValueError("bad source vertex")

    def __del__(self):
        if getattr(self, "h", None):
            lib().ox_destroy(self.h)
            self.h = None

    def step(self, dt: float, nsteps: int = 1):
        lib().ox_step(self.h, dt, nsteps)

    @property
    def y(self) -> np.ndarray:
        out = np.zeros(self.n)
        lib().ox_get_y(self.h, _p(out, C.c_double))
        return out

    @y.setter
    def y(self, v):
        a = np.ascontiguousarray(v, dtype=np.float64)
        lib().ox_set_y(self.h, _p(a, C.c_double))

    @property
    def I(self) -> np.ndarray:
        out = np.zeros((self.n, self.nbins))
        lib().ox_get_I(self.h, _p(out, C.c_double))
        return out

    @I.setter
    def I(self, v):
        a = np.ascontiguousarray(v, dtype=np.float64)
        lib().ox_set_I(self.h, _p(a, C.c_double))

    def photons(self) -> np.ndarray:
        """Photons in flight towards every vertex (any transport)."""
        out = np.zeros(self.n)
        lib().ox_get_inflight(self.h, _p(out, C.c_double))
        return out

    def diffuse(self):
        """(pending, emitted) of diffuse recombination radiation: each cell's
        ground-level recombination photons of the last step, which it emits
        in the next one, and the photons recombining cells have emitted."""
        out = np.zeros(self.n)
        emitted = lib().ox_get_diffuse(self.h, _p(out, C.c_double))
        return out, emitted

    def ballistic(self):
        """(stb nnz x 4, twin nnz, thick n) of ballistic or combined transport:
        the ballistic straight sets, the reverse-edge index and the modes of
        the last step."""
        nnz = int(self._keep["rp"][-1])
        stb = np.zeros((max(nnz, 1), 4), dtype=np.uint8)
        twin = np.zeros(max(nnz, 1), dtype=np.int64)
        thick = np.zeros(self.n, dtype=np.uint8)
        lib().ox_get_ballistic(self.h, _p(stb, C.c_uint8), _p(twin, C.c_int64),
                               _p(thick, C.c_uint8))
        return stb[:nnz], twin[:nnz], thick

    @property
    def budget(self) -> dict:
        out = np.zeros(4)
        lib().ox_get_budget(self.h, _p(out, C.c_double))
        return dict(emitted=out[0], absorbed=out[1], escaped=out[2], in_flight=out[3])

    @property
    def kappa(self) -> float:
        return lib().ox_get_kappa(self.h)

    @property
    def step_count(self) -> int:
        return lib().ox_get_step(self.h)

    @property
    def stats(self) -> dict:
        out = np.zeros(2, dtype=np.int64)
        lib().ox_get_stats(self.h, _p(out, C.c_int64))
        return dict(subcycles=int(out[0]), capped=int(out[1]))

    def vertex_consts(self):
        A, t, R0 = np.zeros(self.n), np.zeros(self.n), np.zeros(self.n)
        lib().ox_get_vertex_consts(self.h, _p(A, C.c_double), _p(t, C.c_double),
                                   _p(R0, C.c_double))
        return A, t, R0

    def tables(self):
        nnz = int(self._keep["rp"][-1])
        q = np.zeros((max(nnz, 1), 3), dtype=np.int32)
        st = np.zeros((max(nnz, 1), 4), dtype=np.uint8)
        ml = np.zeros(self.n)
        lib().ox_get_tables(self.h, _p(q, C.c_int32), _p(st, C.c_uint8), _p(ml, C.c_double))
        return q[:nnz], st[:nnz], ml

    def mark_removal(self, y_thresh: float, min_spacing: float) -> np.ndarray:
        """Vertices the dynamic grid update removes (Sect. 2.1.4), ascending."""
        out = np.zeros(self.n, dtype=np.int32)
        k = lib().ox_mark_removal(self.h, y_thresh, min_spacing, _p(out, C.c_int32))
        return out[:k].copy()

    def rebuild(self, removed, problem_new, old_of_new, params=None):
        """The state after the dynamic update on the re-triangulated survivors:
        photons of removed vertices handed over, neutral fractions, step count,
        budget and sources carried to the new grid (a new OracleSim)."""
        if self.p.transport != 0:
            raise NotImplementedError("the dynamic update carries bins: direction conserving only")
        if self.p.alpha_A > 0:
            raise NotImplementedError("the dynamic update does not carry diffuse photons")
        removed = np.ascontiguousarray(removed, dtype=np.int32)
        I = np.ascontiguousarray(self.I)
        lib().ox_hand_over(self.h, len(removed), _p(removed, C.c_int32), _p(I, C.c_double))
        old_of_new = np.asarray(old_of_new, dtype=np.int64)
        y = self.y[old_of_new]
        new = OracleSim(problem_new, params or self.p, self._keep["bins"], y0=y)
        new.I = np.ascontiguousarray(I[old_of_new])
        lib().ox_set_step(new.h, self.step_count)
        b = np.array([self.budget[k] for k in ("emitted", "absorbed", "escaped", "in_flight")])
        b[3] = float(new.I.sum())
        lib().ox_set_budget(new.h, _p(np.ascontiguousarray(b), C.c_double))
        return new

    def associate_all(self, step: int) -> np.ndarray:
        out = np.zeros((self.n, self.nbins), dtype=np.int32)
        lib().ox_associate_all(self.h, step, _p(out, C.c_int32))
        return out


# ---------------------------------------------------------------------------
# The oracle's own Delaunay builder
# ---------------------------------------------------------------------------
def triangulate(points: np.ndarray) -> np.ndarray:
    """Finite Delaunay tetrahedra (int32 [ntet, 4]) by Bowyer-Watson insertion."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    out = C.POINTER(C.c_int32)()
    nt = lib().dl_triangulate(len(pts), _p(pts, C.c_double), C.byref(out))
    if nt < 0:
        raise ValueError("degenerate point set")
    tets = np.ctypeslib.as_array(out, shape=(nt, 4)).copy() if nt else np.zeros((0, 4), np.int32)
    lib().dl_free(out)
    return tets


def insphere(a, b, c, d, e) -> bool:
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (a, b, c, d, e)]
    return bool(lib().dl_insphere(*[_p(x, C.c_double) for x in arrs]))


def edges_of_tets(tets: np.ndarray) -> set:
    """Undirected edge set {(lo, hi)} of a tetrahedralisation."""
    out = set()
    for t in np.asarray(tets):
        for a in range(4):
            for b in range(a + 1, 4):
                u, v = int(t[a]), int(t[b])
                out.add((min(u, v), max(u, v)))
    return out


# ---------------------------------------------------------------------------
# Analytic Test-1 solutions (Sect. 5.1)
# ---------------------------------------------------------------------------
def stromgren_radius(rate: float, nH: float, alpha_B: float) -> float:
    """Eq. (stromgren_radius): r_S = (3 Ndot / (4 pi alpha_B n_H^2))^(1/3)."""
    return (3.0 * rate / (4.0 * math.pi * alpha_B * nH * nH)) ** (1.0 / 3.0)


def recombination_time(nH: float, alpha_B: float) -> float:
    """t_rec = 1 / (alpha_B n_H)."""
    return 1.0 / (alpha_B * nH)


def ifront_radius(t, rate, nH, alpha_B):
    """Eq. (IFront_pos): r_I(t) = r_S (1 - exp(-t / t_rec))^(1/3)."""
    rs = stromgren_radius(rate, nH, alpha_B)
    tr = recombination_time(nH, alpha_B)
    return rs * (1.0 - np.exp(-np.asarray(t, dtype=np.float64) / tr)) ** (1.0 / 3.0)


def ifront_velocity(t, rate, nH, alpha_B):
    """Eq. (IFront_vel)."""
    rs = stromgren_radius(rate, nH, alpha_B)
    tr = recombination_time(nH, alpha_B)
    e = np.exp(-np.asarray(t, dtype=np.float64) / tr)
    return rs / (3.0 * tr) * e / (1.0 - e) ** (2.0 / 3.0)


def equilibrium_profile(r_max: float, rate: float, nH: float, alpha_B: float, sigma: float,
                        n_r: int = 20000):
    """Neutral fraction y(r) of the equilibrium H II region, Eq. (inner_stromgren_region).

    Monochromatic: n_HI * Ndot e^-tau sigma / (4 pi r^2) = x^2 n_H^2 alpha_B with
    n_HI = y n_H and x = 1 - y, and d tau / dr = n_H sigma y.  At each radius
    the balance is a quadratic in y; tau is integrated with the midpoint rule
    on a fine radial grid.  Returns (r, y, tau).
    """
    r = np.linspace(r_max / n_r, r_max, n_r)
    y = np.zeros(n_r)
    tau = np.zeros(n_r)

    def y_of(rr, tt):
        # y c = (1-y)^2, c = Ndot e^-tau sigma / (4 pi r^2 n_H alpha_B)
        c = rate * math.exp(-tt) * sigma / (4.0 * math.pi * rr * rr * nH * alpha_B)
        # y^2 - (2 + c) y + 1 = 0, root in [0, 1]
        b = 2.0 + c
        return (b - math.sqrt(b * b - 4.0)) / 2.0 if c < 1e12 else 1.0 / c

    t_acc = 0.0
    r_prev = 0.0
    y_prev = 0.0
    for i in range(n_r):
        dr = r[i] - r_prev
        # midpoint: predict y at the midpoint with the current tau
        y_mid = y_of(r_prev + 0.5 * dr, t_acc + 0.5 * dr * nH * sigma * y_prev)
        t_acc += dr * nH * sigma * y_mid
        y[i] = y_of(r[i], t_acc)
        tau[i] = t_acc
        r_prev = r[i]
        y_prev = y[i]
    return r, y, tau


def ifront_position(y, pos, volume, mask, centre, r_max, nshell: int = 56) -> float:
    """I-front position: the outermost radius at which the volume-weighted
    average of the ionised fraction x = 1 - y over spherical shells about
    ``centre`` (width r_max / nshell, vertices in ``mask``) falls through
    0.5, linearly interpolated between shell midpoints; nan if it never
    does."""
    d = np.linalg.norm(np.asarray(pos)[mask] - np.asarray(centre), axis=1)
    x = 1.0 - np.asarray(y)[mask]
    v = np.asarray(volume)[mask]
    edges = np.linspace(0.0, r_max, nshell + 1)
    k = np.digitize(d, edges) - 1
    ok = (k >= 0) & (k < nshell)
    vol = np.bincount(k[ok], weights=v[ok], minlength=nshell)
    xs = np.bincount(k[ok], weights=(x * v)[ok], minlength=nshell) / np.maximum(vol, 1e-300)
    mid = 0.5 * (edges[1:] + edges[:-1])
    for j in range(nshell - 1, 0, -1):
        if xs[j - 1] >= 0.5 > xs[j]:
            return float(mid[j - 1] + (xs[j - 1] - 0.5) / (xs[j - 1] - xs[j]) * (mid[j] - mid[j - 1]))
    return float("nan")


def equilibrium_front(rate: float, nH: float, alpha_B: float, sigma: float) -> float:
    """Radius where the equilibrium profile (Eq. inner_stromgren_region) is
    half ionised."""
    rs = stromgren_radius(rate, nH, alpha_B)
    r, y, _ = equilibrium_profile(2.0 * rs, rate, nH, alpha_B, sigma)
    j = int(np.argmax(y > 0.5))
    return float(r[j - 1] + (0.5 - y[j - 1]) / (y[j] - y[j - 1]) * (r[j] - r[j - 1]))


def ionised_radius_octant(y, volume, interior_mask) -> float:
    """I-front radius of a corner source from the ionised volume of the octant."""
    vi = float(np.sum((1.0 - y[interior_mask]) * volume[interior_mask]))
    return (3.0 * 8.0 * vi / (4.0 * math.pi)) ** (1.0 / 3.0)


def ionised_radius_sphere(y, volume, interior_mask) -> float:
    """I-front radius of a centred source from the ionised volume."""
    vi = float(np.sum((1.0 - y[interior_mask]) * volume[interior_mask]))
    return (3.0 * vi / (4.0 * math.pi)) ** (1.0 / 3.0)
