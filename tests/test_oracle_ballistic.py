"""Pins of the oracle's ballistic and combined transport (Sect. 2.2.2, 2.2.4,
5.1.1, 5.1.3), against what the paper and the mathematics fix:

* combined transport with tau_switch = inf is direction-conserving transport
  everywhere, and with tau_switch = 0 ballistic transport everywhere: the
  results must equal those of the two pure modes;
* the ballistic straight sets follow their definition (the <= 3 most
  straightforward neighbours with respect to the incoming direction, none
  beyond 90 degrees), brute force from the quantised edge directions;
* in a transparent medium photons are only moved: after two steps from a
  source, every vertex holds exactly what the routing rules send it
  (brute force over the source's neighbours);
* the photon budget closes through every conversion between bins and edges;
* a ballistic photon forgets its direction after a few steps (Sect. 2.2.2,
  KPCI09): the mean radius of a source's photons grows ever slower, while
  direction-conserving transport keeps it growing at a constant rate;
* at equilibrium the ionised volume is set by recombinations alone, so the
  I-front of every mode follows the equilibrium solution (Fig.
  IFront_ballistic: within about 1% at 500 Myr).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

DT = 2.5 * I.MYR_S


@pytest.fixture(scope="module")
def small():
    return I.stromgren_problem(2048, seed=1), I.fibonacci_bins(42)


def _sim(prob, bins, **kw):
    return O.OracleSim(prob, O.Params(nbins=len(bins), seed=1, **kw), bins)


def test_combined_reduces_to_the_pure_modes(small):
    prob, bins = small
    dct = _sim(prob, bins)
    thin = _sim(prob, bins, transport=2, tau_switch=math.inf)
    bal = _sim(prob, bins, transport=1)
    thick = _sim(prob, bins, transport=2, tau_switch=0.0)
    mixed = _sim(prob, bins, transport=2, tau_switch=1.0)
    for s in (dct, thin, bal, thick, mixed):
        s.step(DT, 20)
    assert np.array_equal(dct.y, thin.y)
    np.testing.assert_allclose(thin.photons(), dct.photons(), rtol=1e-12, atol=0)
    for k in ("emitted", "absorbed", "escaped"):
        assert thin.budget[k] == dct.budget[k]
    assert np.array_equal(bal.y, thick.y) and bal.budget == thick.budget
    assert np.array_equal(bal.photons(), thick.photons())
    # tau_switch = 1 mixes the modes (the ionised inside is thin) and differs
    # from both pure modes
    n_thick = int(mixed.ballistic()[2].sum())
    assert 0.1 * prob.n < n_thick < 0.9 * prob.n
    assert not np.array_equal(mixed.y, dct.y) and not np.array_equal(mixed.y, bal.y)


def test_ballistic_tables_follow_their_definition(small):
    prob, bins = small
    stb, twin, _ = _sim(prob, bins, transport=1).ballistic()
    q, _, _ = O.edge_tables(prob.pos, prob.row_ptr, prob.col)
    q = q.astype(np.int64)
    for i in range(prob.n):
        r0, r1 = prob.row_ptr[i], prob.row_ptr[i + 1]
        for e in range(r0, r1):
            assert prob.col[twin[e]] == i and prob.row_ptr[prob.col[e]] <= twin[e] < prob.row_ptr[prob.col[e] + 1]
            d = q[r0:r1] @ (-q[e])
            cand = sorted((-int(d[k]), k) for k in range(r1 - r0) if d[k] > 0)[:3]
            assert stb[e, 3] == len(cand)
            assert list(stb[e, :len(cand)]) == [k for _, k in cand]


def test_transparent_routing_two_steps(small):
    """sigma = 0: nothing is absorbed.  Step 1 puts rate dt / deg on every
    in-edge from the source; step 2 moves each of those packets, in equal
    parts, to the neighbours of its ballistic straight set (a sink passes
    nothing on) and the source emits again."""
    prob, bins = small
    s = _sim(prob, bins, transport=1, sigma=0.0)
    stb, twin, _ = s.ballistic()
    v = int(prob.src_vertex[0])
    rate = float(prob.src_rate[0])
    N = rate * DT
    r0, r1 = prob.row_ptr[v], prob.row_ptr[v + 1]
    deg = r1 - r0
    s.step(DT, 1)
    want = np.zeros(prob.n)
    want[prob.col[r0:r1]] = N / deg
    np.testing.assert_allclose(s.photons(), want, rtol=1e-12, atol=0)
    s.step(DT, 1)
    want = np.zeros(prob.n)
    escaped = 0.0
    for e in range(r0, r1):
        w = prob.col[e]
        want[w] += N / deg                       # the second emission
        if prob.flags[w] & 1:
            escaped += N / deg
            continue
        ein = twin[e]                            # the packet sits on w's in-edge from v
        cnt = stb[ein, 3]
        if cnt == 0:
            escaped += N / deg
        for m in range(cnt):
            want[prob.col[prob.row_ptr[w] + stb[ein, m]]] += N / deg / cnt
    np.testing.assert_allclose(s.photons(), want, rtol=1e-12, atol=1e-300)
    b = s.budget
    assert b["absorbed"] == pytest.approx(0.0, abs=1e-9 * b["emitted"])
    assert b["escaped"] == pytest.approx(escaped, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("transport,tau_switch", [(1, 0.0), (2, 1.0), (2, 0.05)])
def test_budget_closes_through_conversions(small, transport, tau_switch):
    prob, bins = small
    s = _sim(prob, bins, transport=transport, tau_switch=tau_switch)
    for _ in range(6):
        s.step(DT, 5)
        b = s.budget
        assert abs(b["emitted"] - b["absorbed"] - b["escaped"] - b["in_flight"]) <= 1e-12 * b["emitted"]
        assert b["in_flight"] == pytest.approx(s.photons().sum(), rel=1e-12)
        y = s.y
        assert y.min() >= 0.0 and y.max() <= 1.0


def test_ballistic_photons_forget_their_direction():
    prob = I.stromgren_problem(16384, seed=3)
    bins = I.fibonacci_bins(84)
    c = prob.pos[prob.src_vertex[0]]
    rv = np.linalg.norm(prob.pos - c, axis=1)
    growth = {}
    for tp in (0, 1):
        s = O.OracleSim(prob, O.Params(nbins=84, seed=0, sigma=0.0, transport=tp), bins)
        radius = []
        for _ in range(12):
            s.step(1e13, 1)
            ph = s.photons()
            radius.append(float((ph * rv).sum() / ph.sum()))
        d = np.diff(radius)
        growth[tp] = d[-3:].mean() / d[:3].mean()
    assert growth[0] > 0.9          # direction conserving: constant speed
    assert growth[1] < 0.8          # ballistic: slows down as directions are lost


@pytest.mark.parametrize("transport,tau_switch", [(1, 0.0), (2, 1.0)])
def test_ifront_follows_equilibrium_solution(transport, tau_switch):
    nH, Nd, a = 1e-3, 5e48, 2.59e-13
    r, ye, _ = O.equilibrium_profile(9 * I.KPC_CM, Nd, nH, a, I.SIGMA_H)
    r_eq = (3 * np.trapezoid((1 - ye) * r * r, r)) ** (1 / 3)
    tr = O.recombination_time(nH, a)
    prob = I.stromgren_problem(8192, seed=0)
    s = O.OracleSim(prob, O.Params(nbins=42, seed=0, transport=transport, tau_switch=tau_switch),
                    I.fibonacci_bins(42))
    steps = 100
    dt = 500 * I.MYR_S / steps
    for k in range(5):
        s.step(dt, steps // 5)
        t = (k + 1) * (steps // 5) * dt
        ratio = O.ionised_radius_sphere(s.y, prob.volume, prob.interior) / (
            r_eq * (1 - math.exp(-t / tr)) ** (1 / 3))
        if t >= 2.4 * tr:
            assert abs(ratio - 1) < 0.03, (t / I.MYR_S, ratio)
    assert abs(ratio - 1) < 0.02
