"""Vertex removal from a Delaunay tetrahedralisation by local re-triangulation:
the host step of the dynamic grid update (Sect. 2.1.4).

Removing a vertex v leaves a cavity, the union of the tetrahedra around v.
Every tetrahedron outside the cavity keeps its empty circumsphere, so it stays
in the Delaunay tetrahedralisation of the remaining points, and so do the
faces on the cavity's boundary.  The tetrahedra that fill the cavity have
their vertices among v's neighbours and empty circumspheres, so (for points in
general position) they are exactly the tetrahedra of the Delaunay
tetrahedralisation of v's neighbours whose interiors lie in the cavity.
Vertices removed together form an independent set (no two adjacent), so no
tetrahedron holds two of them, the cavities have disjoint interiors and each
is filled on its own.

The paper's QHull cannot delete points and rebuilds the whole grid after a
removal; here only the cavities are re-triangulated and the graph, the cell
volumes and the tetrahedra are patched: by the library's native code
(Bowyer-Watson on each vertex's neighbours, threaded; the default), or with
QHull per cavity and numpy patches (``method="qhull"``, the cross-check).
Each cavity's new tetrahedra must fill its volume; a vertex on the convex
hull (whose removal changes the hull) fails that check, and the grid is then
rebuilt from scratch.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


def _in_any_tet(p: np.ndarray, tets: np.ndarray, eps: float = 1e-9) -> np.ndarray:
    """Whether each point p[k] (K x 3) lies in one of the tetrahedra
    (S x 4 x 3), by barycentric coordinates."""
    a = tets[:, 0]
    m = np.stack([tets[:, 1] - a, tets[:, 2] - a, tets[:, 3] - a], axis=-1)  # S x 3 x 3
    minv = np.linalg.inv(m)
    lam = np.einsum("sij,ksj->ksi", minv, p[:, None, :] - a[None, :, :])     # K x S x 3
    ok = (lam >= -eps).all(axis=-1) & (lam.sum(axis=-1) <= 1.0 + eps)
    return ok.any(axis=1)


def _fill_cavities(jobs):
    """New tetrahedra of each cavity (global ids), or None where QHull
    refuses: jobs are (link ids, link positions relative to the removed
    vertex, the star's tetrahedra as relative corner positions)."""
    from scipy.spatial import Delaunay

    out = []
    for link, p, star_xyz in jobs:
        if len(link) < 4:
            out.append(None)
            continue
        try:
            cand = Delaunay(p).simplices
        except Exception:  # QHull refuses (e.g. a flat neighbourhood)
            out.append(None)
            continue
        inside = _in_any_tet(p[cand].mean(axis=1), star_xyz)
        out.append(link[cand[inside]])
    return out


_POOL = None


def _pool(workers: int):
    """Worker processes for the cavities, started once (spawned: the caller
    may already hold a CUDA context, which a forked child must not inherit)."""
    global _POOL
    import concurrent.futures as cf
    import multiprocessing as mp

    if _POOL is None or _POOL._max_workers != workers:
        if _POOL is not None:
            _POOL.shutdown()
        _POOL = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    return _POOL


def remove_vertices(problem: "I.Problem", removed, allow_rebuild: bool = True,
                    workers: int | None = None, method: str = "native") -> tuple:
    """The grid without the `removed` vertices (an independent set of the
    graph): survivors in their old order, their Delaunay graph, cell volumes
    (1/4 of the incident tetrahedra), media, flags, sources and tetrahedra.
    Returns (problem, old_of_new), as a full rebuild of the survivors would.

    Needs the grid's tetrahedra (``problem.simplices``); a grid without them,
    or a cavity that cannot be filled locally, is rebuilt by QHull (or, with
    ``allow_rebuild=False``, raises RuntimeError).

    method="native" (default) runs the whole removal in the library
    (sx_remesh_remove: Bowyer-Watson per cavity, single-pass patches);
    method="qhull" fills the cavities with QHull in `workers` processes
    (default: the host's cores when there are more than 256 cavities) and
    patches the arrays with numpy."""

    def rebuild(why):
        if not allow_rebuild:
            raise RuntimeError(why)
        return I.survivor_problem(problem, np.flatnonzero(rem))

    n = problem.n
    rem = np.zeros(n, dtype=bool)
    rem[np.asarray(removed, dtype=np.int64)] = True
    if problem.simplices is None:
        return rebuild("the grid has no tetrahedra")
    if np.any(rem[problem.src_vertex]):
        raise ValueError("sources are never removed")
    if method == "native":
        from . import simplex as S

        try:
            r = S.sx_remesh_remove(problem.pos, problem.row_ptr, problem.col, problem.simplices,
                                   problem.volume, np.flatnonzero(rem))
        except S.RemeshError as e:
            if e.vertex < 0:
                raise ValueError("removed vertices must not be adjacent") from e
            return rebuild(f"the cavity of vertex {e.vertex} cannot be filled locally")
        keep = r["old_of_new"].astype(np.int64)
        new_of_old = np.full(n, -1, dtype=np.int64)
        new_of_old[keep] = np.arange(len(keep))
        p = I.Problem(pos=np.ascontiguousarray(problem.pos[keep]), row_ptr=r["row_ptr"], col=r["col"],
                      nH=problem.nH[keep].copy(), volume=r["volume"], flags=problem.flags[keep].copy(),
                      src_vertex=new_of_old[problem.src_vertex].astype(np.int32),
                      src_rate=problem.src_rate.copy(), box=problem.box, meta=dict(problem.meta),
                      simplices=r["tets"])
        return p, r["old_of_new"]
    if method != "qhull":
        raise ValueError("method must be 'native' or 'qhull'")
    simp = np.asarray(problem.simplices)
    hit = rem.view(np.uint8)[simp]
    cnt = hit.sum(axis=1, dtype=np.uint8)
    if np.any(cnt > 1):
        raise ValueError("removed vertices must not be adjacent")
    star_ids = np.flatnonzero(cnt == 1)
    st = simp[star_ids].astype(np.int64)
    owner = st[hit[star_ids].astype(bool)]
    order = np.argsort(owner, kind="stable")
    st, owner = st[order], owner[order]
    cuts = np.flatnonzero(np.diff(owner)) + 1
    pos = problem.pos
    vs = owner[np.r_[0, cuts]] if len(owner) else np.zeros(0, dtype=np.int64)
    jobs = []
    for grp, v in zip(np.split(st, cuts), vs):
        link = np.unique(grp[grp != v])
        origin = pos[v]  # coordinates relative to v: better conditioned
        jobs.append((link, pos[link] - origin, pos[grp] - origin))
    if workers is None:
        import os

        workers = min(16, os.cpu_count() or 1) if len(jobs) > 256 else 1
    if workers > 1 and len(jobs) > 1:
        nchunk = min(len(jobs), 4 * workers)
        bounds = np.linspace(0, len(jobs), nchunk + 1).astype(int)
        parts = _pool(workers).map(_fill_cavities, [jobs[i:j] for i, j in zip(bounds[:-1], bounds[1:])])
        filled = [t for part in parts for t in part]
    else:
        filled = _fill_cavities(jobs)
    for t, v in zip(filled, vs):
        if t is None:
            return rebuild(f"the cavity of vertex {int(v)} cannot be filled locally")
    new = np.concatenate(filled) if filled else np.zeros((0, 4), dtype=np.int64)
    # every cavity's new tetrahedra fill its volume (a vertex on the hull does not)
    if len(vs):
        cav_of_new = np.repeat(np.arange(len(vs)), [len(t) for t in filled])
        cav_of_old = np.repeat(np.arange(len(vs)), np.diff(np.r_[0, cuts, len(st)]))
        v_old = np.bincount(cav_of_old, weights=I.tet_volumes(pos, st), minlength=len(vs))
        v_new = np.bincount(cav_of_new, weights=I.tet_volumes(pos, new), minlength=len(vs))
        bad = np.flatnonzero(~(np.abs(v_new - v_old) <= 1e-9 * v_old))
        if len(bad):
            return rebuild(f"the cavity of vertex {int(vs[bad[0]])} cannot be filled locally")

    # the graph: old edges without the removed vertices, plus the cavity
    # tetrahedra's edges not already present (keys src * n + dst, sorted)
    deg = np.diff(problem.row_ptr)
    src = np.repeat(np.arange(n, dtype=np.int32), deg)
    dst = problem.col
    keep_e = ~(rem[src] | rem[dst])
    src, dst = src[keep_e], dst[keep_e]
    key = src.astype(np.int64) * n + dst
    pairs = np.concatenate([new[:, [a, b]] for a, b in
                            ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))])
    add = np.unique(np.concatenate([pairs[:, 0] * n + pairs[:, 1], pairs[:, 1] * n + pairs[:, 0]]))
    at = np.searchsorted(key, add)
    present = (at < len(key)) & (key[np.minimum(at, len(key) - 1)] == add)
    at, add = at[~present], add[~present]
    src = np.insert(src, at, (add // n).astype(np.int32))
    dst = np.insert(dst, at, (add % n).astype(np.int32))

    keep = np.flatnonzero(~rem)
    n2 = len(keep)
    new_of_old = np.full(n, -1, dtype=np.int32)
    new_of_old[keep] = np.arange(n2, dtype=np.int32)
    col2 = new_of_old[dst]
    row_ptr2 = np.zeros(n2 + 1, dtype=np.int64)
    np.cumsum(np.bincount(new_of_old[src], minlength=n2), out=row_ptr2[1:])

    # cell volumes: the cavity's old tetrahedra leave their vertices, the new
    # ones join theirs, a quarter each
    vol = problem.volume.astype(np.float64).copy()
    np.add.at(vol, st.ravel(), -np.repeat(I.tet_volumes(pos, st) * 0.25, 4))
    np.add.at(vol, new.ravel(), np.repeat(I.tet_volumes(pos, new) * 0.25, 4))

    simp2 = np.concatenate([new_of_old[simp[cnt == 0]], new_of_old[new]])
    p = I.Problem(pos=np.ascontiguousarray(pos[keep]), row_ptr=row_ptr2, col=col2,
                  nH=problem.nH[keep].copy(), volume=vol[keep], flags=problem.flags[keep].copy(),
                  src_vertex=new_of_old[problem.src_vertex].astype(np.int32),
                  src_rate=problem.src_rate.copy(), box=problem.box, meta=dict(problem.meta),
                  simplices=simp2)
    return p, keep.astype(np.int32)
