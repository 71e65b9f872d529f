"""Seeded input recipes: the Test-1 grid and the clumpy medium."""
import numpy as np
import pytest

from paper_0912_4273_gb300 import inputs as I


def test_stromgren_grid_shape():
    p = I.stromgren_problem(4096, seed=2)
    inter = p.interior
    assert inter.sum() == 4096
    src = p.src_vertex[0]
    assert np.allclose(p.pos[src], 0.5 * p.box)           # centred source (Sect. 5.1)
    assert np.all((p.pos[inter] >= 0) & (p.pos[inter] <= p.box))
    assert np.all(p.flags[~inter] == I.FLAG_SINK)
    assert p.volume[inter].sum() == pytest.approx(p.box**3, rel=0.02)
    assert np.array_equal(p.pos, I.stromgren_problem(4096, seed=2).pos)  # seeded


def test_gaussian_field_spectrum_and_lognormal_moments():
    d = I.gaussian_random_field(32, -3.0, seed=1)
    assert abs(d.mean()) < 1e-12 and d.std() == pytest.approx(1.0)
    # slope of the measured spectrum (isotropic average) close to -3
    P = np.abs(np.fft.rfftn(d)) ** 2
    k1 = np.fft.fftfreq(32)
    k3 = np.fft.rfftfreq(32)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k3[None, None, :] ** 2)
    sel = (kk > 0.05) & (kk < 0.4)
    slope = np.polyfit(np.log(kk[sel]), np.log(P[sel]), 1)[0]
    assert -3.4 < slope < -2.6
    n = I.lognormal_density(32, 1.5, -3.0, 1e-3, seed=1)
    assert np.log(n).std() == pytest.approx(1.5, rel=1e-6)


def test_clumpy_problem_samples_density_to_the_third():
    p = I.clumpy_problem(20000, mesh=16, nsrc=16, seed=3)
    inter = p.interior
    assert inter.sum() == 20000 and len(p.src_vertex) == 16
    assert np.all((p.src_rate >= 1e47) & (p.src_rate <= 1e49))
    # sources sit at the densest cells
    rho = I.lognormal_density(16, 1.5, -3.0, 1e-3, seed=3)
    assert np.allclose(np.sort(p.nH[p.src_vertex])[::-1], np.sort(rho.ravel())[::-1][:16])
    # point counts per cell follow n^(1/3)
    h = p.box / 16
    ijk = np.clip((p.pos[inter] / h).astype(int), 0, 15)
    cnt = np.bincount(np.ravel_multi_index(ijk.T, (16,) * 3), minlength=16**3)
    w = np.cbrt(rho.ravel())
    assert np.corrcoef(cnt, w)[0, 1] > 0.6


def test_hybrid_sampling_function():
    """Eq. realistic_sampling: the d-th power of n/n0 below the reference
    density, the power alpha above it, 1/2 at n0; Q_n/Q_y (the relation
    below it) is the inverse logarithmic slope of the sampling function."""
    n0, a = 3.69e-5, 0.3
    lo = np.array([1e-4, 1e-3]) * n0
    hi = np.array([1e3, 1e4]) * n0
    np.testing.assert_allclose(I.hybrid_sampling(lo, n0, a), (lo / n0) ** 3, rtol=1e-2)
    np.testing.assert_allclose(I.hybrid_sampling(hi, n0, a), (hi / n0) ** a, rtol=1e-2)
    assert I.hybrid_sampling(n0, n0, a) == pytest.approx(0.5)
    y = np.geomspace(1e-3, 1e3, 25)
    eps = 1e-6
    slope = (np.log(I.hybrid_sampling(y * (1 + eps), 1.0, a)) - np.log(I.hybrid_sampling(y * (1 - eps), 1.0, a))) / (
        np.log(1 + eps) - np.log(1 - eps))
    np.testing.assert_allclose(I.sampling_gradient_ratio(y, a), 1.0 / slope, rtol=1e-6)
    # the limits of that ratio: 1/d well below n0, 1/alpha well above
    assert I.sampling_gradient_ratio(1e-6, a) == pytest.approx(1 / 3, rel=1e-3)
    assert I.sampling_gradient_ratio(1e6, a) == pytest.approx(1 / a, rel=1e-3)


def test_clumpy_problem_with_hybrid_sampling():
    n0 = 1e-3
    p = I.clumpy_problem(20000, mesh=16, nsrc=16, seed=3, sampling="hybrid", alpha=0.3, n0=n0)
    rho = I.lognormal_density(16, 1.5, -3.0, 1e-3, seed=3)
    h = p.box / 16
    ijk = np.clip((p.pos[p.interior] / h).astype(int), 0, 15)
    cnt = np.bincount(np.ravel_multi_index(ijk.T, (16,) * 3), minlength=16**3)
    w = I.hybrid_sampling(rho.ravel(), n0, 0.3)
    assert np.corrcoef(cnt, w)[0, 1] > 0.6
    # low-density cells (below n0, sampled to the third power) hold fewer
    # points than with n^(1/3) sampling
    q = I.clumpy_problem(20000, mesh=16, nsrc=16, seed=3)
    ijk = np.clip((q.pos[q.interior] / h).astype(int), 0, 15)
    cq = np.bincount(np.ravel_multi_index(ijk.T, (16,) * 3), minlength=16**3)
    low = rho.ravel() < 0.1 * n0
    assert cnt[low].sum() < 0.5 * cq[low].sum()
    with pytest.raises(ValueError):
        I.clumpy_problem(1000, mesh=8, sampling="square")
