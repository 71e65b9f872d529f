"""FP32 transport sums every bin's arriving packets with compensation
(Kahan-Babuska: the rounding error of each addition, exact by two-sum, is
carried and added back once all packets are in).

The grid is a fan: 47 senders of degree 1 around one sink.  Every sender is
a transparent source (n_H = 0), so in each step it passes all of its
photons, in every bin, along its only edge to the sink.  Sender 1 emits
2^40 photons/s and the 46 others 0.4 x 2^-24 of that each: every one of
their shares is below half an ulp of the large share, so a plain FP32 sum in
the fixed (edge) order returns the large share alone in every bin, while the
46 small shares together are about 18 ulps.  The photons that reach the sink
("escaped") and the budget's closure then show whether they were kept.  Every
share is exactly representable (rates, dt = 1 s and 32 bins are powers of
two times small integers), so the only rounding is in the sums.
"""
import numpy as np
import pytest

import oracle as O
from paper_0912_4273_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_0912_4273_gb300 import simplex as S  # noqa: E402

K = 47                    # senders
NB = 32                   # bins
BIG = 2.0 ** 40           # photons / s of sender 1
SMALL = 26214.0           # photons / s of each other sender: 0.4 * 2^-24 * BIG, an integer
DT = 1.0                  # s


def fan_problem():
    rng = np.random.default_rng(7)
    n = K + 1
    d = rng.normal(size=(K, 3)) * 0.2 + np.array([1.0, 0.0, 0.0])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pos = np.vstack([np.zeros(3), d]) * 3.0e20
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1] = K
    row_ptr[2:] = K + np.arange(1, K + 1)
    col = np.concatenate([np.arange(1, K + 1), np.zeros(K)]).astype(np.int32)
    flags = np.zeros(n, np.uint8)
    flags[0] = S.SX_FLAG_SINK
    rates = np.full(K, SMALL)
    rates[0] = BIG
    return I.Problem(pos=pos, row_ptr=row_ptr, col=col, nH=np.zeros(n), volume=np.full(n, 1e60),
                     flags=flags, src_vertex=np.arange(1, K + 1, dtype=np.int32), src_rate=rates,
                     box=1.0, meta={})


def plain_fp32_sum_error():
    """Relative error of the escaped photons if every bin summed its packets
    plainly in FP32 (the fixed edge order, sender 1 first)."""
    big, small = np.float32(BIG * DT / NB), np.float32(SMALL * DT / NB)
    acc = big
    for _ in range(K - 1):
        acc = np.float32(acc + small)
    exact = float(big) + (K - 1) * float(small)
    return abs(float(acc) - exact) / exact


def test_small_packets_survive_a_large_one():
    prob = fan_problem()
    bins = I.fibonacci_bins(NB)
    # kappa is fixed (the fan is no Delaunay graph, and n_H = 0 makes it moot)
    ref = O.OracleSim(prob, O.Params(nbins=NB, seed=3, kappa=1.0), bins)
    ref.step(DT, 2)
    rb = ref.budget
    assert rb["absorbed"] == 0.0
    # the test discriminates: plain FP32 sums would lose ~1e-6 of the photons
    assert plain_fp32_sum_error() > 5e-7
    s = S.Solver(bins, precision=S.SX_FP32_TRANSPORT, seed=3, kappa=1.0).load(prob)
    s.step(DT, 2)
    b = s.budget
    s.close()
    # one step's photons reached the sink, the next step's are in flight
    assert b["escaped"] == pytest.approx(rb["escaped"], rel=1.5e-7)
    assert b["in_flight"] == pytest.approx(rb["in_flight"], rel=1.5e-7)
    residual = (b["emitted"] - b["absorbed"] - b["escaped"] - b["in_flight"]) / b["emitted"]
    assert abs(residual) < 1.5e-7, residual
