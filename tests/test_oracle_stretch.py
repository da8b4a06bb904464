"""Pins of the oracle's contrast stretch (Sec. 4: the optional preprocessing
step stretches a frame to [0, 1] with 0.35% saturation).

Each check fixes the oracle against something other than its own code: the
closed form on a ramp, a counting characterisation of the two order
statistics (no sorting), the rank invariants the limits must satisfy, shift
invariance, and the degenerate frames."""
import numpy as np
import pytest

import oracle

SAT = 0.0035


def _limits_by_counting(c, sat):
    """lo = smallest v with #(c <= v) > k, hi = largest v with #(c >= v) > k,
    k = floor(sat/2 n): the same order statistics found by counting."""
    v = np.minimum(c.astype(np.int64).ravel(), 4095)
    n = v.size
    k = int(np.floor(sat * 0.5 * n))
    k = min(k, (n - 1) // 2)
    hist = np.bincount(v, minlength=4096)
    le = np.cumsum(hist)                   # #(c <= v)
    ge = np.cumsum(hist[::-1])[::-1]       # #(c >= v)
    lo = int(np.argmax(le > k))
    hi = int(4095 - np.argmax(ge[::-1] > k))
    return lo, hi


def test_ramp_closed_form():
    n = 4000
    c = np.arange(n, dtype=np.uint16)
    k = int(np.floor(SAT * 0.5 * n))       # 7
    assert oracle.stretch_rank(n, SAT) == k == 7
    lo, hi = oracle.stretch_limits(c, SAT)
    assert (lo, hi) == (k, n - 1 - k)
    out = oracle.stretch(c, lo, hi)
    want = np.clip((np.arange(n, dtype=np.float64) - k) / (n - 1 - 2 * k), 0.0, 1.0).astype(np.float32)
    assert np.array_equal(out, want)
    assert out[k] == 0.0 and out[n - 1 - k] == 1.0


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_limits_equal_counting_definition(seed):
    rng = np.random.default_rng(seed)
    h, w = [(37, 53), (256, 256), (100, 1), (512, 300)][seed]
    # many ties, a few saturated outliers, values past the 12-bit range
    c = rng.poisson(900, size=(h, w)).astype(np.uint16)
    c.ravel()[rng.choice(c.size, size=max(1, c.size // 200), replace=False)] = 4095
    c.ravel()[rng.choice(c.size, size=max(1, c.size // 500), replace=False)] = 5000
    assert oracle.stretch_limits(c, SAT) == _limits_by_counting(c, SAT)


def test_rank_invariants_on_plif_frame():
    from paper_2010_08486_gb300 import synth
    c = synth.plif_frame_u16(synth.PLIF_SEED_BASE, 256, 256)
    lo, hi = oracle.stretch_limits(c, SAT)
    k = oracle.stretch_rank(c.size, SAT)
    v = np.minimum(c.astype(np.int64), 4095)
    assert np.count_nonzero(v < lo) <= k < np.count_nonzero(v <= lo)
    assert np.count_nonzero(v > hi) <= k < np.count_nonzero(v >= hi)
    out = oracle.stretch(c, lo, hi)
    assert out.min() == 0.0 and out.max() == 1.0
    # the map is monotone in the counts
    order = np.argsort(v.ravel(), kind="stable")
    assert np.all(np.diff(out.ravel()[order]) >= 0)
    # the saturated fractions: at most k + ties on each side map to the ends
    assert np.count_nonzero(out == 0.0) == np.count_nonzero(v <= lo)
    assert np.count_nonzero(out == 1.0) == np.count_nonzero(v >= hi)


def test_shift_invariance():
    rng = np.random.default_rng(7)
    c = rng.integers(100, 3000, size=(64, 80)).astype(np.uint16)
    a = oracle.preprocess(c, SAT)
    b = oracle.preprocess(c + 500, SAT)
    assert np.array_equal(a, b)


def test_degenerate_frames():
    c = np.full((16, 16), 1234, dtype=np.uint16)
    assert oracle.stretch_limits(c, SAT) == (1234, 1234)
    assert not np.any(oracle.preprocess(c, SAT))
    one = np.array([[17]], dtype=np.uint16)
    assert oracle.stretch_limits(one, SAT) == (17, 17)
    # two values: k = 0 for small frames, limits are the extremes
    c = np.array([[3, 9]], dtype=np.uint16)
    assert oracle.stretch_limits(c, SAT) == (3, 9)
    assert oracle.preprocess(c, SAT).tolist() == [[0.0, 1.0]]
    # counts above the 12-bit range act as 4095
    c = np.array([[0, 4095, 60000]], dtype=np.uint16)
    assert oracle.preprocess(c, SAT).tolist() == [[0.0, 1.0, 1.0]]
