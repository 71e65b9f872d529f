"""Pins of the oracle's dynamic grid update (Sect. 2.1.4): which vertices go,
where their photons go, and that the solve carries on consistently."""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

DT = 2.5 * I.MYR_S


@pytest.fixture(scope="module")
def lit():
    prob = I.stromgren_problem(4096, seed=11)
    sim = O.OracleSim(prob, O.Params(nbins=42, seed=11), I.fibonacci_bins(42))
    sim.step(DT, 80)
    return prob, sim


def test_removed_vertices_form_the_local_minimum_independent_set(lit):
    prob, sim = lit
    _, _, ml = sim.tables()
    thr, spacing = 1e-2, np.median(ml) * 1.2
    rem = sim.mark_removal(thr, spacing)
    assert len(rem) > 10 and np.all(np.diff(rem) > 0)
    y = sim.y
    src = set(prob.src_vertex.tolist())
    cand = np.array([(not prob.flags[i] & 1) and i not in src and y[i] < thr and ml[i] < spacing
                     for i in range(prob.n)])
    rs = set(rem.tolist())
    for i in range(prob.n):
        nb = prob.col[prob.row_ptr[i]:prob.row_ptr[i + 1]]
        lower = [j for j in nb if cand[j] and j < i]
        assert (i in rs) == (bool(cand[i]) and not lower)
        if i in rs:
            assert not any(j in rs for j in nb)  # independent


def test_hand_over_conserves_photons_and_budget(lit):
    prob, sim = lit
    _, _, ml = sim.tables()
    rem = sim.mark_removal(1e-2, np.median(ml) * 1.2)
    newp, o2n = I.survivor_problem(prob, rem)
    b0 = sim.budget
    new = sim.rebuild(rem, newp, o2n, params=O.Params(nbins=42, seed=11, kappa=sim.kappa))
    assert new.I.sum() == pytest.approx(sim.I.sum(), rel=1e-13)
    assert new.step_count == sim.step_count
    assert np.array_equal(new.y, sim.y[o2n])
    b1 = new.budget
    for k in ("emitted", "absorbed", "escaped"):
        assert b1[k] == b0[k]
    new.step(DT, 20)
    b = new.budget
    assert abs(b["emitted"] - b["absorbed"] - b["escaped"] - b["in_flight"]) < 1e-10 * b["emitted"]


def test_front_survives_the_removal():
    """Removing ionised vertices above the minimum resolution keeps the
    equilibrium I-front close to the one on the full grid (Sect. 5.1.1)."""
    prob = I.stromgren_problem(8192, seed=0)
    bins = I.fibonacci_bins(42)
    full = O.OracleSim(prob, O.Params(nbins=42), bins)
    full.step(DT, 200)
    r_full = O.ionised_radius_sphere(full.y, prob.volume, prob.interior)
    sim = O.OracleSim(prob, O.Params(nbins=42), bins)
    p = prob
    _, _, ml = sim.tables()
    spacing = np.median(ml) * 1.1
    for _ in range(4):
        sim.step(DT, 50)
        rem = sim.mark_removal(1e-3, spacing)
        p2, o2n = I.survivor_problem(p, rem)
        sim = sim.rebuild(rem, p2, o2n)
        p = p2
    assert p.n < prob.n
    r = O.ionised_radius_sphere(sim.y, p.volume, p.interior)
    assert abs(r / r_full - 1) < 0.05
