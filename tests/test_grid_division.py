"""The batch kernels form the grid values t_j = fl32(j) / fl32(n - 1) without
a division for n - 1 < 2^16: q0 = RN(j r) with r = RN(1 / (n - 1)), then
q1 = RN(q0 + RN(j - q0 (n - 1)) r) (Markstein's reciprocal-based division
with one fused correction step).  This checks, in FP32 emulated with exact
FP64 steps, that q1 is the IEEE quotient: exhaustively for n - 1 < 2^11 and
on a random sample below 2^16 (the full range below 2^16, 2.1e9 pairs, was
checked the same way while building it).  The outer fused step is emulated
as RN32(RN64(.)); that equals RN32 of the exact value unless the FP64 value
is an FP32 midpoint, which the check rules out case by case."""
import numpy as np


def _check(d, j):
    df = np.float32(d)
    r = np.float32(1.0) / df
    j = j.astype(np.float32)
    q0 = j * r
    res = (j.astype(np.float64) - q0.astype(np.float64) * float(df)).astype(np.float32)  # exact, then RN32
    v = q0.astype(np.float64) + res.astype(np.float64) * float(r)
    q1 = v.astype(np.float32)
    lo = np.nextafter(q1, np.float32(-np.inf)).astype(np.float64)
    hi = np.nextafter(q1, np.float32(np.inf)).astype(np.float64)
    q1d = q1.astype(np.float64)
    assert not np.any((v == (q1d + lo) / 2) | (v == (q1d + hi) / 2)), d
    np.testing.assert_array_equal(q1, j / df)


def test_reciprocal_division_exhaustive_small():
    for d in range(1, 1 << 11):
        _check(d, np.arange(d + 1))


def test_reciprocal_division_sampled_below_2_16():
    rng = np.random.default_rng(11)
    for d in rng.integers(1 << 11, 1 << 16, size=300):
        d = int(d)
        _check(d, np.unique(np.concatenate([rng.integers(0, d + 1, size=4000), [0, 1, d - 1, d]])))
