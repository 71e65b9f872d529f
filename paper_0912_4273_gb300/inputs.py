"""Seeded synthetic inputs for the SimpleX2 DCT sweep.

This module builds the *inputs* of the transport path and nothing else: point
sets (the point process of Sect. 2.1.1), the Delaunay graph of those points
(Sect. 2.1.2; QHull, as in the paper, through ``scipy.spatial.Delaunay``),
per-vertex volumes, the global direction-bin table and the source list.  It
holds none of the transport, absorption or chemistry arithmetic; the CUDA
library and the CPU oracle both take what is built here as plain arrays.

Every generator is seeded (numpy ``PCG64``) so that a (recipe, seed) pair gives
the same arrays on every machine.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Unit conversions (cgs).
KPC_CM = 3.0856775814913673e21
MYR_S = 3.15576e13

# Physical constants of Test 1 (Sect. 5.1): case-B recombination at 1e4 K and
# the hydrogen photoionisation cross-section at 13.6 eV (Eq. for sigma_H).
ALPHA_B = 2.59e-13
SIGMA_H = 6.3e-18

FLAG_SINK = 1


# --------------------------------------------------------------------------
# Ordering helpers
# --------------------------------------------------------------------------
def _spread_bits_21(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_keys(points: np.ndarray, lo=None, hi=None, bits: int = 21) -> np.ndarray:
    """63-bit Morton (Z-order) keys of points in the box [lo, hi]^3."""
    p = np.asarray(points, dtype=np.float64)
    lo = p.min(axis=0) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = p.max(axis=0) if hi is None else np.asarray(hi, dtype=np.float64)
    scale = (2**bits - 1) / np.maximum(hi - lo, 1e-300)
    q = np.clip(((p - lo) * scale).astype(np.int64), 0, 2**bits - 1)
    return (_spread_bits_21(q[:, 0]) | (_spread_bits_21(q[:, 1]) << np.uint64(1))
            | (_spread_bits_21(q[:, 2]) << np.uint64(2)))


def morton_order(points: np.ndarray, lo=None, hi=None) -> np.ndarray:
    """Permutation that sorts points along a Morton curve (stable)."""
    return np.argsort(morton_keys(points, lo, hi), kind="stable")


# --------------------------------------------------------------------------
# Delaunay graph
# --------------------------------------------------------------------------
@dataclasses.dataclass
class DelaunayGraph:
    row_ptr: np.ndarray   # int64 [n+1]
    col: np.ndarray       # int32 [nnz], rows sorted ascending, symmetric
    volume: np.ndarray    # float64 [n]; 1/4 of the incident tetrahedron volumes
    simplices: np.ndarray  # int32 [ntet, 4]


def csr_from_simplices(n: int, simplices: np.ndarray):
    """Symmetric CSR (rows sorted ascending) of the edge set of tetrahedra."""
    s = np.asarray(simplices, dtype=np.int64)
    pairs = np.concatenate([s[:, [a, b]] for a, b in
                            ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))])
    lo_ = np.minimum(pairs[:, 0], pairs[:, 1])
    hi_ = np.maximum(pairs[:, 0], pairs[:, 1])
    key = np.unique(lo_ * n + hi_)
    a = key // n
    b = key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src = src[order]
    dst = dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, dst.astype(np.int32)


def tet_volumes(points: np.ndarray, simplices: np.ndarray) -> np.ndarray:
    p = points[simplices]
    d1 = p[:, 1] - p[:, 0]
    d2 = p[:, 2] - p[:, 0]
    d3 = p[:, 3] - p[:, 0]
    return np.abs(np.einsum("ij,ij->i", d1, np.cross(d2, d3))) / 6.0


def delaunay_graph(points: np.ndarray) -> DelaunayGraph:
    """Delaunay tetrahedralisation by QHull (the package the paper uses)."""
    from scipy.spatial import Delaunay

    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = len(pts)
    tri = Delaunay(pts)
    simp = tri.simplices.astype(np.int32)
    row_ptr, col = csr_from_simplices(n, simp)
    tv = tet_volumes(pts, simp)
    vol = np.zeros(n, dtype=np.float64)
    for c in range(4):
        np.add.at(vol, simp[:, c], tv * 0.25)
    return DelaunayGraph(row_ptr=row_ptr, col=col, volume=vol, simplices=simp)


# --------------------------------------------------------------------------
# Direction bins
# --------------------------------------------------------------------------
def fibonacci_bins(nbins: int, ordered: bool = True) -> np.ndarray:
    """nbins unit vectors on a Fibonacci lattice (float64 [nbins, 3]).

    z_j = 1 - (2j+1)/n, phi_j = j * pi * (3 - sqrt 5).  With ``ordered`` the
    vectors are permuted along a Morton curve of the unit cube so that bins
    with neighbouring indices point in neighbouring directions.
    """
    j = np.arange(nbins, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / nbins
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = j * math.pi * (3.0 - math.sqrt(5.0))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    if ordered:
        d = d[morton_order(d, lo=[-1, -1, -1], hi=[1, 1, 1])]
    return np.ascontiguousarray(d)


# --------------------------------------------------------------------------
# Problems
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """One SimpleX2 grid with its medium and sources (all arrays host numpy)."""

    pos: np.ndarray        # float64 [n, 3], cm
    row_ptr: np.ndarray    # int64 [n+1]
    col: np.ndarray        # int32 [nnz]
    nH: np.ndarray         # float64 [n], cm^-3
    volume: np.ndarray     # float64 [n], cm^3
    flags: np.ndarray      # uint8 [n], bit0 = sink
    src_vertex: np.ndarray  # int32 [nsrc]
    src_rate: np.ndarray   # float64 [nsrc], photons / s
    box: float             # cm, side of the interior cube [0, box]^3
    meta: dict
    simplices: np.ndarray | None = None  # int32 [ntet, 4], the Delaunay tetrahedra

    @property
    def n(self) -> int:
        return len(self.pos)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def interior(self) -> np.ndarray:
        return (self.flags & FLAG_SINK) == 0


def _sink_shell(rng, n_interior: int, box: float, margin_spacings: float):
    """Poisson points of the interior density in a margin around [0, box]^3."""
    spacing = box / n_interior ** (1.0 / 3.0)
    m = margin_spacings * spacing
    outer = box + 2.0 * m
    n_outer = rng.poisson(n_interior * (outer / box) ** 3)
    c = rng.random((n_outer, 3)) * outer - m
    inside = np.all((c >= 0.0) & (c <= box), axis=1)
    return c[~inside]


def stromgren_problem(n_interior: int = 8192, box_kpc: float = 13.2, nH: float = 1e-3,
                      rate: float = 5e48, seed: int = 0, margin_spacings: float = 1.5,
                      corner_source: bool = False) -> Problem:
    """Isothermal H II region expansion (Test 1) on a Poisson-Delaunay grid.

    ``n_interior`` vertices fill [0, L]^3 (one of them is the source, at the
    centre of the box as in Sect. 5.1, or at the corner (0,0,0)), and a sink
    shell of the same point density surrounds the cube; photons that reach a
    sink leave the volume.  Vertices are stored in Morton order.

    The default geometry is the paper's: a 13.2 kpc box with the source at its
    centre, which is the mirror-symmetric completion of a corner source in a
    6.6 kpc cube.  (A sink boundary through a corner source removes the
    photons that the symmetry planes would keep.)
    """
    rng = np.random.default_rng(seed)
    L = box_kpc * KPC_CM
    src_pos = np.zeros(3) if corner_source else np.full(3, 0.5 * L)
    interior = np.concatenate([src_pos[None, :], rng.random((n_interior - 1, 3)) * L])
    shell = _sink_shell(rng, n_interior, L, margin_spacings)
    pts = np.concatenate([interior, shell])
    flags = np.zeros(len(pts), dtype=np.uint8)
    flags[n_interior:] = FLAG_SINK
    order = morton_order(pts)
    pts = np.ascontiguousarray(pts[order])
    flags = flags[order]
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    g = delaunay_graph(pts)
    return Problem(pos=pts, row_ptr=g.row_ptr, col=g.col,
                   nH=np.full(len(pts), nH, dtype=np.float64), volume=g.volume, flags=flags,
                   src_vertex=np.array([inv[0]], dtype=np.int32),
                   src_rate=np.array([rate], dtype=np.float64), box=L,
                   meta=dict(kind="stromgren", n_interior=n_interior, box_kpc=box_kpc, nH=nH,
                             rate=rate, seed=seed, corner_source=corner_source),
                   simplices=g.simplices)


def cached(recipe, *args, cache_dir: str | None = None, **kw) -> Problem:
    """``recipe(*args, **kw)``, memoised as an .npz in ``cache_dir`` (or in the
    directory named by $SX_GRID_CACHE; no caching if neither is set)."""
    import hashlib
    import json
    import os

    cache_dir = cache_dir or os.environ.get("SX_GRID_CACHE")
    if not cache_dir:
        return recipe(*args, **kw)
    key = hashlib.sha1(json.dumps([recipe.__name__, args, kw], sort_keys=True, default=str)
                       .encode()).hexdigest()[:16]
    path = os.path.join(cache_dir, f"grid_{key}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return Problem(pos=z["pos"], row_ptr=z["row_ptr"], col=z["col"], nH=z["nH"],
                       volume=z["volume"], flags=z["flags"], src_vertex=z["src_vertex"],
                       src_rate=z["src_rate"], box=float(z["box"]),
                       meta=json.loads(str(z["meta"])),
                       simplices=z["simplices"] if "simplices" in z.files else None)
    p = recipe(*args, **kw)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    extra = {} if p.simplices is None else {"simplices": p.simplices}
    np.savez(tmp, pos=p.pos, row_ptr=p.row_ptr, col=p.col, nH=p.nH, volume=p.volume,
             flags=p.flags, src_vertex=p.src_vertex, src_rate=p.src_rate, box=p.box,
             meta=json.dumps(p.meta), **extra)
    os.replace(tmp, path)
    return p


def gaussian_random_field(mesh: int, slope: float = -3.0, seed: int = 0) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field on a periodic mesh^3
    with power spectrum P(k) ~ k^slope (white noise shaped in Fourier space)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((mesh, mesh, mesh))
    k1 = np.fft.fftfreq(mesh)
    k3 = np.fft.rfftfreq(mesh)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k3[None, None, :] ** 2)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (slope / 2.0)
    f = np.fft.irfftn(np.fft.rfftn(white) * amp, s=white.shape, axes=(0, 1, 2))
    f -= f.mean()
    return f / f.std()


def lognormal_density(mesh: int = 128, sigma_ln: float = 1.5, slope: float = -3.0,
                      nbar: float = 1e-3, seed: int = 0) -> np.ndarray:
    """n = nbar exp(sigma delta - sigma^2 / 2) of a Gaussian field delta."""
    d = gaussian_random_field(mesh, slope, seed)
    return nbar * np.exp(sigma_ln * d - 0.5 * sigma_ln**2)


def hybrid_sampling(n, n0, alpha: float, d: int = 3):
    """The sampling function of Eq. realistic_sampling: the harmonic mean of
    (n/n0)^d and (n/n0)^alpha, so that densities below the reference n0 are
    sampled to the d-th power (edge length proportional to the mean free
    path, Eq. delaunay_vs_mfp) and those above it to the power alpha < d
    (not undersampling the low-density regions)."""
    y = np.asarray(n, dtype=np.float64) / n0
    return 1.0 / (y ** (-float(d)) + y ** (-float(alpha)))


def sampling_gradient_ratio(y, alpha: float, d: int = 3):
    """Q_n / Q_y of the hybrid sampling at y = n / n0 (the relation below
    Eq. realistic_sampling): how much flatter the point density is than the
    medium density."""
    y = np.asarray(y, dtype=np.float64)
    return (y ** (-alpha) + y ** (-float(d))) / (y * (alpha * y ** (-alpha - 1.0) + d * y ** (-d - 1.0)))


def clumpy_problem(n_points: int = 1 << 22, mesh: int = 128, box_kpc: float = 13.2,
                   nbar: float = 1e-3, sigma_ln: float = 1.5, nsrc: int = 16, seed: int = 0,
                   margin_spacings: float = 1.5, sampling: str = "cbrt", alpha: float = 0.3,
                   n0: float | None = None) -> Problem:
    """Clumpy medium: a lognormal density on a mesh^3 grid, vertices drawn with
    probability ~ n^(1/3) per cell (or, with sampling="hybrid", the paper's
    hybrid sampling function of n with reference density n0, default nbar,
    and power alpha) and placed uniformly inside their cell
    (n_H of the cell, nearest grid point), a sink shell around the box, and
    nsrc sources at the centres of the nsrc densest cells with rates
    log-uniform in [1e47, 1e49] photons/s."""
    rng = np.random.default_rng(seed + 7)
    rho = lognormal_density(mesh, sigma_ln, -3.0, nbar, seed)
    L = box_kpc * KPC_CM
    h = L / mesh
    if sampling == "cbrt":
        w = np.cbrt(rho).ravel()
    elif sampling == "hybrid":  # Eq. realistic_sampling with d = 3
        w = hybrid_sampling(rho, nbar if n0 is None else n0, alpha).ravel()
    else:
        raise ValueError("sampling must be 'cbrt' or 'hybrid'")
    counts = rng.multinomial(n_points - nsrc, w / w.sum())
    cell = np.repeat(np.arange(mesh**3), counts)
    ijk = np.stack(np.unravel_index(cell, (mesh,) * 3), axis=1)
    pts = (ijk + rng.random((len(cell), 3))) * h
    dens = np.argsort(rho.ravel())[::-1][:nsrc]
    sijk = np.stack(np.unravel_index(dens, (mesh,) * 3), axis=1)
    spts = (sijk + 0.5) * h
    interior = np.concatenate([spts, pts])
    nh_int = np.concatenate([rho.ravel()[dens], rho.ravel()[cell]])
    shell = _sink_shell(rng, n_points, L, margin_spacings)
    allp = np.concatenate([interior, shell])
    nh = np.concatenate([nh_int, np.full(len(shell), nbar)])
    flags = np.zeros(len(allp), dtype=np.uint8)
    flags[len(interior):] = FLAG_SINK
    order = morton_order(allp)
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    allp = np.ascontiguousarray(allp[order])
    g = delaunay_graph(allp)
    rates = 10.0 ** rng.uniform(47.0, 49.0, nsrc)
    return Problem(pos=allp, row_ptr=g.row_ptr, col=g.col, nH=nh[order], volume=g.volume,
                   flags=flags[order], src_vertex=inv[:nsrc].astype(np.int32), src_rate=rates,
                   box=L, meta=dict(kind="clumpy", n_points=n_points, mesh=mesh, box_kpc=box_kpc,
                                    nbar=nbar, sigma_ln=sigma_ln, nsrc=nsrc, seed=seed,
                                    sampling=sampling, alpha=alpha, n0=n0),
                   simplices=g.simplices)


def shadow_problem(n_interior: int = 64 ** 3, seed: int = 0, contrast: float = 200.0,
                   slab_pc=(855.0, 2138.0, 2138.0), distance_pc: float = 1096.0,
                   **stromgren_kw) -> Problem:
    """Shadowing behind a dense clump (Test 2 of Sect. 5.2): the Test-1 grid
    and source, with a uniform rectangular slab `contrast` times denser than
    its surroundings, `slab_pc` in size (x, y, z), its near face
    `distance_pc` from the source along +x and centred on the source's line
    of sight.  The paper prints the sizes in kpc, which cannot fit a
    13.2 kpc box: they are read as pc.  The grid is sampled uniformly, as in
    Test 1."""
    p = stromgren_problem(n_interior, seed=seed, **stromgren_kw)
    c = p.pos[p.src_vertex[0]]
    pc = KPC_CM / 1e3
    lo = c + np.array([distance_pc * pc, -0.5 * slab_pc[1] * pc, -0.5 * slab_pc[2] * pc])
    hi = lo + np.array(slab_pc) * pc
    inside = np.all((p.pos >= lo) & (p.pos <= hi), axis=1) & p.interior
    nH = p.nH.copy()
    nH[inside] *= contrast
    meta = dict(p.meta, kind="shadow", contrast=contrast, slab_pc=list(slab_pc),
                distance_pc=distance_pc, slab_lo=lo.tolist(), slab_hi=hi.tolist())
    return dataclasses.replace(p, nH=nH, meta=meta)


def survivor_problem(problem: Problem, removed) -> tuple:
    """The grid of the vertices that survive a removal (Sect. 2.1.4): the
    survivors in their old order, re-triangulated by QHull, with their media,
    flags and sources.  Returns (problem, old_of_new)."""
    rem = np.zeros(problem.n, dtype=bool)
    rem[np.asarray(removed, dtype=np.int64)] = True
    keep = np.nonzero(~rem)[0]
    new_of_old = np.full(problem.n, -1, dtype=np.int64)
    new_of_old[keep] = np.arange(len(keep))
    pts = np.ascontiguousarray(problem.pos[keep])
    g = delaunay_graph(pts)
    assert np.all(new_of_old[problem.src_vertex] >= 0), "sources are never removed"
    p = Problem(pos=pts, row_ptr=g.row_ptr, col=g.col, nH=problem.nH[keep].copy(),
                volume=g.volume, flags=problem.flags[keep].copy(),
                src_vertex=new_of_old[problem.src_vertex].astype(np.int32),
                src_rate=problem.src_rate.copy(), box=problem.box, meta=dict(problem.meta),
                simplices=g.simplices)
    return p, keep.astype(np.int32)


def point_process_problem(points: np.ndarray, nH, sink_mask=None, sources=()) -> Problem:
    """Wrap an explicit point set (tests): Delaunay graph + uniform volumes."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    g = delaunay_graph(pts)
    flags = np.zeros(len(pts), dtype=np.uint8)
    if sink_mask is not None:
        flags[np.asarray(sink_mask, dtype=bool)] = FLAG_SINK
    nh = np.broadcast_to(np.asarray(nH, dtype=np.float64), (len(pts),)).copy()
    sv = np.array([s for s, _ in sources], dtype=np.int32)
    sr = np.array([r for _, r in sources], dtype=np.float64)
    return Problem(pos=pts, row_ptr=g.row_ptr, col=g.col, nH=nh, volume=g.volume, flags=flags,
                   src_vertex=sv, src_rate=sr, box=float(np.ptp(pts, axis=0).max()),
                   meta=dict(kind="points"), simplices=g.simplices)
