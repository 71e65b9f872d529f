"""Pins of the oracle's random rotation (Sect. 2.2.3: rotating the solid angles).

* Philox4x32-10 against the published known-answer vectors.
* The rotation built from it is orthonormal with determinant +1 and Haar
  distributed (first and second moments), with the rejection rate of a
  uniform point in the 4-ball.
* The bin map after a rotation sends each old bin to its closest new bin.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLDEN, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert list(O.philox4x32_10(ctr, key)) == out


def test_rotation_is_proper_orthonormal():
    for s in range(500):
        R, att = O.rotation(12345, s)
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
        assert 1 <= att <= 64


def test_rotation_is_haar():
    n = 4000
    Rs = np.array([O.rotation(7, s)[0] for s in range(n)])
    atts = np.array([O.rotation(7, s)[1] for s in range(n)])
    # E[R_ij] = 0 and E[R_ij^2] = 1/3 for a uniformly random rotation
    se = 1.0 / math.sqrt(3.0 * n)
    assert np.abs(Rs.mean(axis=0)).max() < 5 * se
    assert np.abs((Rs**2).mean(axis=0) - 1.0 / 3.0).max() < 0.03
    # rotated z axis uniform on the sphere: E[z]=0, E[z^2]=1/3 per component
    z = Rs[:, :, 2]
    assert np.abs(z.mean(axis=0)).max() < 5 * se
    # acceptance of a uniform point of the 4-cube inside the unit 4-ball: pi^2/32
    p_acc = math.pi**2 / 32.0
    assert abs(1.0 / atts.mean() - p_acc) < 0.02


def test_rotation_depends_on_seed_and_step():
    a = O.rotation(0, 3)[0]
    assert not np.allclose(a, O.rotation(1, 3)[0])
    assert not np.allclose(a, O.rotation(0, 4)[0])
    assert np.array_equal(a, O.rotation(0, 3)[0])


def test_rotated_bins_quantisation():
    bins = I.fibonacci_bins(84)
    R, _ = O.rotation(0, 11)
    q = O.rotated_bins(R, bins)
    u = bins @ R.T
    # |q - 127 u| <= 1/2 (+ rounding of u); quantised vectors stay near unit length
    assert np.abs(q - 127.0 * u).max() <= 0.5 + 1e-9
    ln = np.linalg.norm(q, axis=1)
    assert np.all(np.abs(ln - 127.0) < 1.5)


def test_bin_map_closest_and_identity():
    bins = I.fibonacci_bins(42)
    R0, _ = O.rotation(3, 0)
    R1, _ = O.rotation(3, 1)
    q0 = O.rotated_bins(R0, bins)
    q1 = O.rotated_bins(R1, bins)
    m = O.bin_map(q0, q1)
    # brute force: exact integer dots, ties -> lowest index
    for b in range(42):
        d = q1.astype(np.int64) @ q0[b].astype(np.int64)
        assert m[b] == int(np.argmax(d))
    assert np.array_equal(O.bin_map(q0, q0), np.arange(42))
    # the map keeps directions: mean angle between old and new bin is small
    cosang = np.einsum("ij,ij->i", q0[np.arange(42)] / 127.0, q1[m] / 127.0)
    assert cosang.min() > 0.8
