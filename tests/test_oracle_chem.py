"""Pins of the oracle's subcycled photoionisation / recombination update.

Sect. 4.5 (Eqs. rate_eq, rate_eq_subcycle, phot_ion_rate_subcycle): at
constant ionising flux over the transfer step the rate equation is integrated
in subcycles; each absorbed photon ionises one atom (photon conservation),
recombinations follow alpha_B n_e n_HII (on-the-spot, Sect. 4.2).
"""
import math

import numpy as np
import pytest

import oracle as O

ALPHA = 2.59e-13
NH = 1e-3
R0 = ALPHA * NH


def test_pure_recombination_matches_closed_form():
    """F = 0: dx/dt = -R0 x^2, x(t) = x0 / (1 + R0 x0 t)."""
    x0 = 0.8
    # a step much shorter than the recombination time: one explicit subcycle
    dt = 0.01 / (R0 * x0)
    y1, f, nsub, _ = O.chem(1 - x0, 0.0, dt, 1e60, 1.0, R0)
    exact = x0 / (1 + R0 * x0 * dt)
    err = abs((1 - y1) - exact)
    assert nsub == 1
    assert err < 1.5 * x0 * (R0 * x0 * dt) ** 2  # second-order local error of one Euler step
    # a long step: subcycling converges at first order in the subcycle fraction
    dt = 5.0 / (R0 * x0)
    exact = x0 / (1 + R0 * x0 * dt)
    errs = []
    for fc in (0.08, 0.04, 0.02):
        y1, _, nsub, _ = O.chem(1 - x0, 0.0, dt, 1e60, 1.0, R0, fc=fc, tol=0.0, max_sub=10**6)
        errs.append(abs((1 - y1) - exact))
    assert errs[2] < 0.02 * exact
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


@pytest.mark.parametrize("tau_max", [1e-4, 0.3, 5.0, 60.0])
@pytest.mark.parametrize("N_in", [1e50, 1e57, 1e59])
def test_each_absorbed_photon_ionises_one_atom(tau_max, N_in):
    """No recombination: N_in (1 - f) = A (y0 - y1)."""
    A = 1e58
    dt = 3e13
    y0 = 0.9
    y1, f, nsub, capped = O.chem(y0, N_in, dt, A, tau_max, 0.0, max_sub=100000)
    assert 0.0 <= f <= 1.0 and 0.0 <= y1 <= y0
    absorbed = N_in * (1.0 - f)
    assert absorbed == pytest.approx(A * (y0 - y1), rel=1e-9, abs=1e-12 * A)


def test_optically_thin_equilibrium_is_the_quadratic_root():
    """Constant Gamma (thin cell): Gamma y = R0 (1 - y)^2 at equilibrium."""
    tau_max = 1e-7
    A = 1.0
    gamma = 1e-12
    F = gamma * A / tau_max
    dt = 1e15  # gamma dt = 1000 e-folds
    y1, f, nsub, capped = O.chem(1.0, F * dt, dt, A, tau_max, R0)
    # y^2 - (2 + g) y + 1 = 0 with g = gamma / R0
    g = gamma / R0
    y_eq = ((2 + g) - math.sqrt((2 + g) ** 2 - 4)) / 2
    assert capped == 0
    assert abs(y1 - y_eq) / y_eq < 1e-4
    # already at equilibrium: one subcycle, state kept
    y2, _, nsub2, _ = O.chem(y1, F * dt, dt, A, tau_max, R0)
    assert nsub2 == 1
    assert abs(y2 - y1) <= 1e-5 * y1


def test_photon_starved_thick_cell_absorbs_everything():
    A = 1e60
    N_in = 1e55
    y1, f, _, _ = O.chem(1.0, N_in, 1e13, A, 50.0, R0)
    assert f < 1e-20
    assert (1.0 - y1) == pytest.approx(N_in / A, rel=1e-9)


def test_random_inputs_stay_physical():
    rng = np.random.default_rng(0)
    for _ in range(300):
        y0 = rng.random()
        N_in = 10 ** rng.uniform(40, 62)
        A = 10 ** rng.uniform(50, 60)
        tau_max = 10 ** rng.uniform(-6, 2)
        dt = 10 ** rng.uniform(11, 15)
        y1, f, nsub, _ = O.chem(y0, N_in, dt, A, tau_max, R0)
        assert 0.0 <= y1 <= 1.0
        assert 0.0 <= f <= 1.0
        assert nsub >= 1


def test_no_photons_no_ions_is_a_fixed_point():
    y1, f, nsub, _ = O.chem(1.0, 0.0, 1e13, 1e58, 3.0, R0)
    assert y1 == 1.0 and nsub == 1


def test_empty_cell_is_transparent():
    """n_H = 0: tau = n_H sigma dL = 0 (Eq. optical_depth), nothing absorbed."""
    y1, f, nsub, _ = O.chem(0.7, 1e55, 1e13, 0.0, 0.0, 0.0)
    assert f == 1.0 and y1 == 0.7 and nsub == 0
