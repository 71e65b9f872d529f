"""Pins of the oracle's own Delaunay builder and of the grids the inputs use.

Sect. 2.1.2: a valid Delaunay triangulation has no point inside any
circumsphere; Poisson-Delaunay vertices have on average 48 pi^2/35 + 2 ~ 15.54
neighbours and edges of mean length ~1.237 n_p^(-1/3).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _brute_force_tets(p):
    n = len(p)
    out = []
    for c in itertools.combinations(range(n), 4):
        a, b, cc, d = (p[i] for i in c)
        vol = np.dot(b - a, np.cross(cc - a, d - a))
        if abs(vol) < 1e-12:
            continue
        if all(not O.insphere(a, b, cc, d, p[e]) for e in range(n) if e not in c):
            out.append(tuple(sorted(c)))
    return sorted(out)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_empty_circumsphere_brute_force(seed):
    p = np.random.default_rng(seed).random((11 + seed, 3))
    mine = sorted(tuple(sorted(int(v) for v in t)) for t in O.triangulate(p))
    assert mine == _brute_force_tets(p)


def test_insphere_predicate():
    a, b, c, d = np.eye(3)[0], np.eye(3)[1], np.eye(3)[2], np.zeros(3)
    assert O.insphere(a, b, c, d, np.array([0.25, 0.25, 0.25]))
    assert not O.insphere(a, b, c, d, np.array([2.0, 2.0, 2.0]))
    # orientation-independent
    assert O.insphere(b, a, c, d, np.array([0.25, 0.25, 0.25]))


def test_matches_qhull_and_fills_hull():
    from scipy.spatial import ConvexHull, Delaunay

    p = np.random.default_rng(5).random((2000, 3))
    tets = O.triangulate(p)
    assert O.edges_of_tets(tets) == O.edges_of_tets(Delaunay(p).simplices)
    v = np.abs(np.einsum("ij,ij->i", p[tets[:, 1]] - p[tets[:, 0]],
                         np.cross(p[tets[:, 2]] - p[tets[:, 0]], p[tets[:, 3]] - p[tets[:, 0]]))) / 6
    assert abs(v.sum() - ConvexHull(p).volume) < 1e-12


def test_poisson_delaunay_statistics():
    g = json.load(open(os.path.join(GOLDEN, "poisson_delaunay.json")))
    n = 20000
    p = np.random.default_rng(9).random((n, 3))
    tets = O.triangulate(p)
    edges = np.array(sorted(O.edges_of_tets(tets)))
    deg = np.bincount(edges.ravel(), minlength=n)
    # vertices far from the boundary: their neighbourhoods are unaffected by the hull
    core = np.all((p > 0.2) & (p < 0.8), axis=1)
    assert abs(deg[core].mean() - g["E_degree_3d"]) < 0.2
    both = core[edges[:, 0]] & core[edges[:, 1]]
    L = np.linalg.norm(p[edges[both, 0]] - p[edges[both, 1]], axis=1)
    # The printed closed form of E(L) lacks its Gamma(1/3) factor; the quoted value
    # 1.237 matches neither the edge-weighted mean (~1.27) nor the simplex-weighted
    # mean (~1.23) of a sample to better than ~3 %, so this pin is loose.
    assert abs(L.mean() / n ** (-1.0 / 3.0) - g["E_length_3d_coeff"]) < 0.05


def test_generator_grid_is_delaunay():
    prob = I.stromgren_problem(2048, seed=3)
    tets = O.triangulate(prob.pos)
    mine = O.edges_of_tets(tets)
    rp, col = prob.row_ptr, prob.col
    gen = {(min(i, int(j)), max(i, int(j))) for i in range(prob.n) for j in col[rp[i]:rp[i + 1]]}
    assert mine == gen
    # symmetric, sorted rows, no self loops
    for i in range(prob.n):
        row = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and i not in row
