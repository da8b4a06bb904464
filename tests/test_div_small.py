"""The ingest's quotient v / d (v / 4095 for 12-bit counts, (c - lo) / (hi - lo)
for the contrast stretch) is formed on the device as q = RN(v rd) with
rd = RN(1/d), then one FMA correction with the exact remainder (Markstein's
final step).  Checked here against the correctly rounded quotient for every
count 0..4095 and every divisor 1..4095, emulating each single-precision step
exactly (products and sums of the correction are exact in double except where
a double result sits on a single-precision midpoint; none does)."""
import numpy as np


def _steps(n, d):
    r = (np.float64(1.0) / d.astype(np.float64)).astype(np.float32)          # RN(1/d)
    q = (n.astype(np.float64) * r.astype(np.float64)).astype(np.float32)     # RN(n rd)
    rem = n.astype(np.float64) - q.astype(np.float64) * d.astype(np.float64)  # exact in double
    s = rem * r.astype(np.float64) + q.astype(np.float64)                    # the correction FMA
    out = s.astype(np.float32)
    # a double that is exactly a float32 midpoint could round differently from
    # the single rounding of the FMA: count them (must be none)
    gap = np.abs(s - out.astype(np.float64))
    mid = np.count_nonzero((gap > 0) & (gap == np.spacing(np.abs(out)).astype(np.float64) / 2))
    return out, mid


def test_reciprocal_of_4095_is_the_rounded_one():
    assert np.float32(1.0) / np.float32(4095.0) == np.float32(1.0 / 4095.0)


def test_quotient_is_correctly_rounded_for_every_count_and_divisor():
    n = np.arange(4096, dtype=np.float32)
    bad = mids = 0
    for d in range(1, 4096):
        dd = np.full(4096, d, np.float32)
        got, mid = _steps(n, dd)
        want = (n.astype(np.float64) / d).astype(np.float32)   # correctly rounded (53 >= 2*24 + 2)
        bad += int(np.count_nonzero(got != want))
        mids += mid
    assert mids == 0 and bad == 0
