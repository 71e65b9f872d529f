"""Pins of the oracle's diffuse recombination radiation (Sect. 2.2.1, 4.5):
case A recombination, and one ionising photon per recombination straight to
the ground level, re-emitted by its cell in every direction bin in the next
step.  The paper's own tests use the on-the-spot approximation instead
(case B, the ground-level photons assumed absorbed where they are made).

* With alpha_A = alpha_B no recombination reaches the ground level, and the
  sweep is the on-the-spot sweep bit for bit.
* The chemistry's recombination count: with no equilibrium hold,
  A dy = recombinations - absorbed photons, to rounding.
* In a transparent medium the emitted photons equal the ground-level
  fraction of the recombinations (A dy), and one recombining cell puts an
  equal share in every bin.
* Ballistic and combined transport (Sect. 2.2.2, 2.2.4): a ballistic cell
  sends its re-emitted photons to all its neighbours in equal parts (the
  scattering transport of Sect. 2.2.1); combined transport with
  tau_switch = inf / 0 is the direction-conserving / ballistic sweep bit
  for bit.
* On the Test-1 grid (Sect. 5.1) the re-emitted photons are absorbed in the
  H II region and its shell.  Case A with re-emission therefore settles at
  the case-B (on-the-spot) I-front, while case A without it settles at the
  smaller case-A front.  In equilibrium the cells re-emit
  (alpha_A - alpha_B) / alpha_B photons per source photon.
"""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

ALPHA_B = 2.59e-13  # case B at 10^4 K (the paper's Test-1 value)
ALPHA_A = 4.18e-13  # case A at 10^4 K (the standard value for the same temperature)
GROUND = (ALPHA_A - ALPHA_B) / ALPHA_A


def test_alpha_A_equal_to_alpha_B_is_the_on_the_spot_sweep():
    p = I.stromgren_problem(2000, seed=3)
    bins = I.fibonacci_bins(42)
    a = O.OracleSim(p, O.Params(nbins=42, seed=3), bins)
    b = O.OracleSim(p, O.Params(nbins=42, seed=3, alpha_A=ALPHA_B), bins)
    for s in (a, b):
        s.step(2.5 * I.MYR_S, 30)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.I, b.I) and a.budget == b.budget
    pending, emitted = b.diffuse()
    assert emitted == 0.0 and not pending.any()


def test_fewer_recombinations_than_case_B_are_refused():
    p = I.stromgren_problem(500, seed=1)
    with pytest.raises(ValueError):
        O.OracleSim(p, O.Params(nbins=21, alpha_A=0.5 * ALPHA_B), I.fibonacci_bins(21))


@pytest.mark.parametrize("N_in_per_atom", [0.0, 1e-3, 0.3, 3.0])
@pytest.mark.parametrize("tau_max", [0.1, 10.0])
def test_chemistry_counts_recombinations(N_in_per_atom, tau_max):
    nH, V = 1e-3, (0.6 * I.KPC_CM) ** 3
    A = nH * V
    N_in = N_in_per_atom * A
    dt = 10 * I.MYR_S
    y0 = 0.3
    # without the equilibrium hold every subcycle changes y by exactly its
    # recombinations minus its ionisations
    y, f, rec, _, _ = O.chem_rec(y0, N_in, dt, A, tau_max, ALPHA_A * nH, tol=0.0)
    scale = max(A * rec, (1 - f) * N_in)
    assert abs(A * (y - y0) - (A * rec - (1 - f) * N_in)) <= 1e-13 * scale
    # the same step as ox_chem
    assert O.chem(y0, N_in, dt, A, tau_max, ALPHA_A * nH, tol=0.0)[:2] == (y, f)
    # with the hold at the last subcycle's rates the balance is kept to the
    # equilibrium tolerance
    y, f, rec, _, _ = O.chem_rec(y0, N_in, dt, A, tau_max, ALPHA_A * nH, tol=1e-5)
    assert abs(A * (y - y0) - (A * rec - (1 - f) * N_in)) <= 1e-5 * scale
    if N_in == 0.0:  # pure recombination: one Euler subcycle, R0 x^2 dt
        assert rec == pytest.approx(ALPHA_A * nH * (1 - y0) ** 2 * dt, rel=1e-15)


def _transparent(p, y0, transport=0):
    return O.OracleSim(p, O.Params(nbins=42, seed=7, sigma=0.0, alpha_A=ALPHA_A, chem_tol=0.0,
                                   transport=transport), I.fibonacci_bins(42), y0=y0)


@pytest.mark.parametrize("transport", [0, 1])
def test_transparent_medium_emits_every_ground_level_recombination(transport):
    p = I.stromgren_problem(2000, rate=0.0, seed=4)
    y0 = np.where(p.interior, 0.5, 1.0)
    s = _transparent(p, y0, transport)
    A = p.nH * p.volume
    for steps in (1, 4, 10):
        s.step(2.5 * I.MYR_S, steps)
        pending, emitted = s.diffuse()
        made = GROUND * np.sum(A * (s.y - y0))  # recombinations = A dy: nothing is absorbed
        assert emitted + pending.sum() == pytest.approx(made, rel=1e-12)
        assert not pending[~p.interior].any()
        b = s.budget
        assert b["emitted"] == pytest.approx(emitted, rel=1e-14)
        assert abs(b["absorbed"]) <= 1e-12 * b["emitted"]
        assert b["escaped"] + b["in_flight"] == pytest.approx(b["emitted"], rel=1e-12)


def test_one_recombining_cell_fills_every_bin():
    p = I.stromgren_problem(2000, rate=0.0, seed=4)
    i = int(np.flatnonzero(p.interior)[100])
    y0 = np.ones(p.n)
    y0[i] = 0.5
    s = _transparent(p, y0)
    s.step(2.5 * I.MYR_S, 1)  # the cell recombines; nothing moves yet
    pending, emitted = s.diffuse()
    D = pending[i]
    assert emitted == 0.0 and D > 0 and np.count_nonzero(pending) == 1
    assert D == pytest.approx(GROUND * p.nH[i] * p.volume[i] * (s.y[i] - 0.5), rel=1e-13)
    assert not s.I.any()
    s.step(2.5 * I.MYR_S, 1)  # emitted: one edge further, an equal share in every bin
    I_ = s.I
    assert np.allclose(I_.sum(axis=0), D / 42, rtol=1e-13, atol=0)
    nbr = set(p.col[p.row_ptr[i]:p.row_ptr[i + 1]].tolist())
    assert set(np.flatnonzero(I_.sum(axis=1)).tolist()) <= nbr  # only i's neighbours hold photons
    assert s.diffuse()[1] == D


def test_one_recombining_ballistic_cell_sends_to_every_neighbour():
    p = I.stromgren_problem(2000, rate=0.0, seed=4)
    i = int(np.flatnonzero(p.interior)[100])
    y0 = np.ones(p.n)
    y0[i] = 0.5
    s = _transparent(p, y0, transport=1)
    s.step(2.5 * I.MYR_S, 1)
    D = s.diffuse()[0][i]
    assert D == pytest.approx(GROUND * p.nH[i] * p.volume[i] * (s.y[i] - 0.5), rel=1e-13)
    s.step(2.5 * I.MYR_S, 1)
    nbr = p.col[p.row_ptr[i]:p.row_ptr[i + 1]]
    got = s.photons()
    assert np.allclose(got[nbr], D / len(nbr), rtol=1e-13, atol=0)
    assert got.sum() == pytest.approx(D, rel=1e-13)


def test_combined_limits_with_diffuse_radiation():
    p = I.stromgren_problem(2000, seed=6)
    bins = I.fibonacci_bins(42)
    runs = {}
    for name, kw in (("dct", dict(transport=0)), ("comb_inf", dict(transport=2, tau_switch=np.inf)),
                     ("bal", dict(transport=1)), ("comb_0", dict(transport=2, tau_switch=0.0))):
        s = O.OracleSim(p, O.Params(nbins=42, seed=6, alpha_A=ALPHA_A, **kw), bins)
        s.step(2.5 * I.MYR_S, 40)
        runs[name] = (s.y, s.budget, s.photons(), s.diffuse())
    for a, b in (("dct", "comb_inf"), ("bal", "comb_0")):
        ya, ba, pa, (da, ea) = runs[a]
        yb, bb, pb, (db, eb) = runs[b]
        assert np.array_equal(ya, yb) and np.array_equal(da, db) and ea == eb and ea > 0
        for k in ("emitted", "absorbed", "escaped"):
            assert ba[k] == bb[k]
        # photons in flight are summed per bin by one sweep and per in-edge
        # by the other
        np.testing.assert_allclose(pb, pa, rtol=1e-12, atol=0)
        assert bb["in_flight"] == pytest.approx(ba["in_flight"], rel=1e-12)


def _equilibrium(p, runs, **common):
    dt = 10 * I.MYR_S
    out = {}
    for name, kw in runs:
        s = O.OracleSim(p, O.Params(nbins=42, seed=0, **common, **kw), I.fibonacci_bins(42))
        s.step(dt, 180)
        e0 = s.diffuse()[1]
        s.step(dt, 20)
        rate = (s.diffuse()[1] - e0) / (20 * dt)
        out[name] = dict(r=O.ionised_radius_sphere(s.y, p.volume, p.interior), diffuse_rate=rate,
                         budget=s.budget)
    return out


@pytest.fixture(scope="module")
def test1_equilibrium():
    """Test 1 (Sect. 5.1) run to 2 Gyr, 16 case-B recombination times, three
    ways: case B on the spot, case A with re-emission, case A without."""
    p = I.stromgren_problem(8192, seed=0)
    return p, _equilibrium(p, (("B", {}), ("A+diffuse", dict(alpha_A=ALPHA_A)),
                               ("A", dict(alpha_B=ALPHA_A))))


def _r_eq(alpha):
    r, y, _ = O.equilibrium_profile(9 * I.KPC_CM, 5e48, 1e-3, alpha, I.SIGMA_H)
    return (3 * np.trapezoid((1 - y) * r * r, r)) ** (1 / 3)


def test_re_emission_restores_the_case_B_front(test1_equilibrium):
    p, out = test1_equilibrium
    for o in out.values():
        b = o["budget"]
        assert abs(b["emitted"] - b["absorbed"] - b["escaped"] - b["in_flight"]) < 1e-10 * b["emitted"]
    assert abs(out["A+diffuse"]["r"] / out["B"]["r"] - 1) < 0.01
    # without re-emission the front settles where case-A recombinations balance the source
    expect = _r_eq(ALPHA_A) / _r_eq(ALPHA_B)
    assert 0.84 < expect < 0.87
    assert abs(out["A"]["r"] / out["B"]["r"] / expect - 1) < 0.02


def test_equilibrium_re_emission_rate(test1_equilibrium):
    """In equilibrium the source's photons plus the re-emitted ones balance
    the case-A recombinations, of which the ground-level fraction is
    re-emitted: D = (alpha_A - alpha_B) / alpha_B * Ndot."""
    p, out = test1_equilibrium
    ndot = float(p.src_rate[0])
    expect = (ALPHA_A - ALPHA_B) / ALPHA_B
    assert abs(out["A+diffuse"]["diffuse_rate"] / ndot / expect - 1) < 0.02
    assert out["B"]["diffuse_rate"] == 0.0 and out["A"]["diffuse_rate"] == 0.0


def test_combined_transport_re_emission_restores_the_case_B_front():
    """The same with combined transport (tau_switch = 1, Sect. 5.1.3): the
    neutral shell beyond the front is ballistic, so re-emitted photons that
    reach it are absorbed by ballistic cells and those made there leave them
    to all neighbours."""
    p = I.stromgren_problem(4096, seed=0)
    out = _equilibrium(p, (("B", {}), ("A+diffuse", dict(alpha_A=ALPHA_A))), transport=2,
                       tau_switch=1.0)
    b = out["A+diffuse"]["budget"]
    assert abs(b["emitted"] - b["absorbed"] - b["escaped"] - b["in_flight"]) < 1e-10 * b["emitted"]
    assert abs(out["A+diffuse"]["r"] / out["B"]["r"] - 1) < 0.015
    rate = out["A+diffuse"]["diffuse_rate"] / float(p.src_rate[0])
    assert abs(rate / ((ALPHA_A - ALPHA_B) / ALPHA_B) - 1) < 0.03

