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


def test_refused_combinations():
    p = I.stromgren_problem(500, seed=1)
    bins = I.fibonacci_bins(21)
    with pytest.raises(ValueError):  # fewer recombinations than case B
        O.OracleSim(p, O.Params(nbins=21, alpha_A=0.5 * ALPHA_B), bins)
    with pytest.raises(ValueError):  # diffuse radiation is direction conserving only
        O.OracleSim(p, O.Params(nbins=21, alpha_A=ALPHA_A, transport=1), bins)


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


def _transparent(p, y0):
    return O.OracleSim(p, O.Params(nbins=42, seed=7, sigma=0.0, alpha_A=ALPHA_A, chem_tol=0.0),
                       I.fibonacci_bins(42), y0=y0)


def test_transparent_medium_emits_every_ground_level_recombination():
    p = I.stromgren_problem(2000, rate=0.0, seed=4)
    y0 = np.where(p.interior, 0.5, 1.0)
    s = _transparent(p, y0)
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


@pytest.fixture(scope="module")
def test1_equilibrium():
    """Test 1 (Sect. 5.1) run to 2 Gyr, 16 case-B recombination times, three
    ways: case B on the spot, case A with re-emission, case A without."""
    p = I.stromgren_problem(8192, seed=0)
    dt = 10 * I.MYR_S
    out = {}
    for name, kw in (("B", {}), ("A+diffuse", dict(alpha_A=ALPHA_A)), ("A", dict(alpha_B=ALPHA_A))):
        s = O.OracleSim(p, O.Params(nbins=42, seed=0, **kw), I.fibonacci_bins(42))
        s.step(dt, 180)
        e0 = s.diffuse()[1]
        s.step(dt, 20)
        rate = (s.diffuse()[1] - e0) / (20 * dt)
        out[name] = dict(r=O.ionised_radius_sphere(s.y, p.volume, p.interior), diffuse_rate=rate,
                         budget=s.budget)
    return p, out


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
