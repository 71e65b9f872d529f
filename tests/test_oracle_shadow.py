"""Pins of the oracle on the shadowing test (Test 2, Sect. 5.2): a point
source irradiates a slab 200 times denser than its surroundings.

* The ionisation front is trapped in the slab and a shadow forms behind it:
  the shadowed region inside the Stromgren radius stays mostly neutral away
  from the shadow's edge (the front penetrates a few cells into it, as the
  paper finds), while the mirror region on the far side of the source, at
  the same distances, is ionised.
* Direction-conserving transport casts a sharper shadow than ballistic
  transport, whose photons forget their direction (Sect. 2.2.2).
"""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I


def shadow_regions(p, margin_cells):
    """Vertices in the slab's geometric shadow (behind it, inside 0.85 r_S,
    at least margin_cells cells inside the shadow cone), and the same region
    mirrored through the source."""
    lo, hi = np.array(p.meta["slab_lo"]), np.array(p.meta["slab_hi"])
    c = p.pos[p.src_vertex[0]]
    d = p.pos - c
    rs = O.stromgren_radius(5e48, 1e-3, 2.59e-13)
    cell = p.box / int(p.meta["n_interior"]) ** (1 / 3)
    near, far = lo[0] - c[0], hi[0] - c[0]
    half_y, half_z = 0.5 * (hi[1] - lo[1]), 0.5 * (hi[2] - lo[2])
    out = []
    for sign in (1, -1):
        x = sign * d[:, 0]
        r = (x > far + cell) & (np.linalg.norm(d, axis=1) < 0.85 * rs) & p.interior
        r &= np.abs(d[:, 1]) < half_y * x / near - margin_cells * cell
        r &= np.abs(d[:, 2]) < half_z * x / near - margin_cells * cell
        out.append(r)
    return out


@pytest.fixture(scope="module")
def runs():
    p = I.shadow_problem(32 ** 3, seed=0)
    y = {}
    for tp in (0, 1):
        s = O.OracleSim(p, O.Params(nbins=42, seed=0, transport=tp), I.fibonacci_bins(42))
        s.step(2.5 * I.MYR_S, 200)  # 500 Myr
        y[tp] = s.y
    return p, y


def test_slab_casts_a_shadow(runs):
    p, y = runs
    slab = p.nH > 1e-3
    assert slab.sum() > 30 and np.median(y[0][slab]) > 0.9  # the front is trapped in the slab
    shadow, mirror = shadow_regions(p, 4)
    assert shadow.sum() > 100
    ion = y[0] < 0.5
    assert ion[mirror].mean() > 0.95
    assert ion[shadow].mean() < 0.35


def test_direction_conserving_shadow_is_sharper_than_ballistic(runs):
    p, y = runs
    shadow, _ = shadow_regions(p, 4)
    assert (y[1][shadow] < 0.5).mean() > (y[0][shadow] < 0.5).mean() + 0.08
