"""The oracle's threaded direction-conserving sweep (used to time the oracle
on every host core) gives the serial sweep's results bit for bit: neutral
fractions, photons in flight per bin, the budget and the diffuse photons,
with sinks, several sources and case-A re-emission on."""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I


@pytest.mark.parametrize("alpha_A", [0.0, 4.18e-13])
def test_threaded_sweep_equals_the_serial_sweep(alpha_A):
    prob = I.stromgren_problem(3000, seed=3)
    bins = I.fibonacci_bins(42)
    dt = 2.5 * I.MYR_S
    p = O.Params(nbins=42, seed=3, alpha_A=alpha_A)
    a = O.OracleSim(prob, p, bins)
    b = O.OracleSim(prob, p, bins, threads=4)
    for k in range(3):
        a.step(dt, 7)
        b.step(dt, 7)
        assert np.array_equal(a.y, b.y)
        assert np.array_equal(a.I, b.I)
        assert a.budget == b.budget
        if alpha_A:
            assert np.array_equal(a.diffuse()[0], b.diffuse()[0])
            assert a.diffuse()[1] == b.diffuse()[1]


def test_threaded_sweep_with_clumpy_medium_and_16_sources():
    prob = I.clumpy_problem(4000, seed=2)
    bins = I.fibonacci_bins(21)
    p = O.Params(nbins=21, seed=2)
    a = O.OracleSim(prob, p, bins)
    b = O.OracleSim(prob, p, bins, threads=3)
    a.step(0.5 * I.MYR_S, 12)
    b.step(0.5 * I.MYR_S, 12)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.I, b.I) and a.budget == b.budget
