"""Vertex removal by local re-triangulation (the host step of the dynamic
grid update, Sect. 2.1.4) against a full QHull rebuild of the survivors: for
points in general position the Delaunay tetrahedralisation is unique, so the
graph must be identical, the cell volumes equal to rounding and the
tetrahedra the same set."""
import numpy as np
import pytest

from paper_0912_4273_gb300 import inputs as I
from paper_0912_4273_gb300 import remesh as R


def _independent_interior(p, k, seed):
    """k interior non-source vertices, no two adjacent (random greedy)."""
    rng = np.random.default_rng(seed)
    ok = p.interior.copy()
    ok[p.src_vertex] = False
    taken = np.zeros(p.n, dtype=bool)
    blocked = np.zeros(p.n, dtype=bool)
    for v in rng.permutation(np.flatnonzero(ok)):
        if blocked[v]:
            continue
        taken[v] = True
        blocked[v] = True
        blocked[p.col[p.row_ptr[v]:p.row_ptr[v + 1]]] = True
        if taken.sum() == k:
            break
    return np.flatnonzero(taken)


def _canon(simp):
    s = np.sort(np.asarray(simp, dtype=np.int64), axis=1)
    return s[np.lexsort(s.T[::-1])]


def _same_grid(a, b):
    assert np.array_equal(a.row_ptr, b.row_ptr)
    assert np.array_equal(a.col, b.col)
    np.testing.assert_allclose(a.volume, b.volume, rtol=1e-11, atol=0)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.flags, b.flags)
    assert np.array_equal(a.nH, b.nH) and np.array_equal(a.src_vertex, b.src_vertex)
    assert np.array_equal(_canon(a.simplices), _canon(b.simplices))


@pytest.mark.parametrize("method", ["native", "qhull"])
@pytest.mark.parametrize("make", [lambda: I.stromgren_problem(3000, seed=21),
                                  lambda: I.clumpy_problem(4000, mesh=16, nsrc=4, seed=2)])
def test_local_removal_equals_full_rebuild(make, method):
    p = make()
    for rnd in range(2):  # twice: the second removal starts from the patched tetrahedra
        rem = _independent_interior(p, 150, seed=rnd)
        assert len(rem) == 150
        full, o2n_full = I.survivor_problem(p, rem)
        loc, o2n = R.remove_vertices(p, rem, allow_rebuild=False, method=method)  # every cavity local
        assert np.array_equal(o2n, o2n_full)
        _same_grid(loc, full)
        # the volume of the cells is conserved
        assert abs(loc.volume.sum() - p.volume.sum()) <= 1e-12 * p.volume.sum()
        p = loc


def test_removal_rules():
    p = I.stromgren_problem(1000, seed=3)
    # adjacent vertices cannot be removed together
    v = int(np.flatnonzero(p.interior)[5])
    w = int(p.col[p.row_ptr[v]])
    with pytest.raises(ValueError):
        R.remove_vertices(p, [v, w])
    with pytest.raises(ValueError):
        R.remove_vertices(p, p.src_vertex)
    # nothing removed: the same grid
    q, o2n = R.remove_vertices(p, [])
    assert np.array_equal(o2n, np.arange(p.n)) and np.array_equal(q.col, p.col)
    # a vertex on the convex hull changes the hull: rebuilt from scratch,
    # with the same result as the full rebuild
    from scipy.spatial import ConvexHull

    hull_v = int(ConvexHull(p.pos).vertices[0])
    for method in ("native", "qhull"):
        with pytest.raises(RuntimeError):
            R.remove_vertices(p, [hull_v], allow_rebuild=False, method=method)
    q, o2n = R.remove_vertices(p, [hull_v])
    full, o2n_full = I.survivor_problem(p, [hull_v])
    assert np.array_equal(o2n, o2n_full)
    _same_grid(q, full)
    # a grid without its tetrahedra is rebuilt as well
    p.simplices = None
    rem = _independent_interior(p, 20, seed=9)
    with pytest.raises(RuntimeError):
        R.remove_vertices(p, rem, allow_rebuild=False)
    q, _ = R.remove_vertices(p, rem)
    full, _ = I.survivor_problem(p, rem)
    _same_grid(q, full)


def test_worker_processes_give_the_same_grid():
    """The QHull method in worker processes equals it in this process."""
    p = I.stromgren_problem(3000, seed=22)
    rem = _independent_interior(p, 300, seed=5)
    a, oa = R.remove_vertices(p, rem, allow_rebuild=False, workers=1, method="qhull")
    b, ob = R.remove_vertices(p, rem, allow_rebuild=False, workers=2, method="qhull")
    assert np.array_equal(oa, ob)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.volume, b.volume) and np.array_equal(a.simplices, b.simplices)
