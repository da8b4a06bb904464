"""The precision/recall harness (host logic): disc overlap against numerical
integration, and the greedy VOC matching on hand-built cases."""
import math

import numpy as np
import pytest

from paper_2010_08486_gb300 import quality


def _grid_intersection(d, r1, r2, n=1500):
    lo, hi = -r1 - 1e-9, max(r1, d + r2) + 1e-9
    xs = np.linspace(lo, hi, n)
    ys = np.linspace(-max(r1, r2), max(r1, r2), n)
    X, Y = np.meshgrid(xs, ys)
    inside = (X * X + Y * Y <= r1 * r1) & ((X - d) ** 2 + Y * Y <= r2 * r2)
    return inside.mean() * (hi - lo) * 2 * max(r1, r2)


@pytest.mark.parametrize("d,r1,r2", [(0.0, 3.0, 3.0), (2.0, 3.0, 3.0), (5.0, 3.0, 4.0), (1.0, 5.0, 2.0),
                                     (6.9, 3.0, 4.0), (7.5, 3.0, 4.0)])
def test_intersection_against_integration(d, r1, r2):
    got = float(quality.disc_intersection(d, r1, r2))
    want = _grid_intersection(d, r1, r2)
    assert abs(got - want) <= 0.01 * math.pi * min(r1, r2) ** 2 + 1e-9


def test_iou_special_cases():
    assert quality.disc_iou(0, 0, 4, 0, 0, 4) == pytest.approx(1.0)
    assert quality.disc_iou(0, 0, 4, 20, 0, 4) == 0.0
    assert quality.disc_iou(1, 1, 2, 1, 1, 4) == pytest.approx(0.25)     # concentric: (r/R)^2


def test_match_hand_cases():
    gt = np.array([[10, 10, 4], [40, 10, 4], [70, 70, 6]], float)
    det = np.array([[10.5, 10, 4], [10, 10.5, 4], [40, 10, 8], [100, 100, 3]], float)
    # the first two detections compete for circle 0: the higher score wins,
    # the other is a false positive; circle 1's detection is too large
    # (IoU 0.25); the last detection meets nothing
    m = quality.match(det, [0.9, 0.95, 0.8, 0.7], gt)
    assert (m.tp, m.fp, m.fn) == (1, 3, 2)
    assert m.pairs.tolist() == [[1, 0]]
    assert m.precision == pytest.approx(0.25) and m.recall == pytest.approx(1 / 3)
    # a detection takes the circle it overlaps most
    gt2 = np.array([[0, 0, 5], [3, 0, 5]], float)
    m2 = quality.match(np.array([[2.8, 0, 5]], float), [1.0], gt2)
    assert m2.pairs.tolist() == [[0, 1]]
    # empty inputs
    assert quality.match(np.zeros((0, 3)), [], gt).recall == 0.0
    assert quality.match(det, [1, 1, 1, 1], np.zeros((0, 3))).precision == 0.0
    # radii from sigma
    c = quality.blob_circles([1], [2], [3.0])
    assert c[0, 2] == pytest.approx(3 * math.sqrt(2))
