"""Detection quality: PASCAL-VOC-style precision and recall of a blob list
against ground-truth circles.  Sec. 5 of arXiv 2010.08486 compares the GPU and
CPU detectors by the precision and recall they reach on synthetic frames.

A detection (x, y, r = sqrt(2) sigma, Sec. 4) matches a ground-truth circle
when the intersection over union of the two discs is at least `iou`
(0.5, the VOC criterion).  Detections are visited by decreasing response;
each takes the still unmatched circle it overlaps most, if any reaches the
criterion (a true positive), otherwise it is a false positive; circles left
unmatched are false negatives.  Host-side numpy; no detector arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def disc_intersection(d, r1, r2):
    """Area of the intersection of two discs of radii r1, r2 whose centres are
    d apart (arrays broadcast): the two circular segments cut by the common
    chord; one disc inside the other gives the smaller disc's area."""
    d = np.asarray(d, np.float64)
    r1 = np.asarray(r1, np.float64)
    r2 = np.asarray(r2, np.float64)
    d, r1, r2 = np.broadcast_arrays(d, r1, r2)
    out = np.zeros(d.shape)
    inside = d <= np.abs(r1 - r2)
    out[inside] = math.pi * np.minimum(r1, r2)[inside] ** 2
    lens = (~inside) & (d < r1 + r2)
    if np.any(lens):
        dd, a, b = d[lens], r1[lens], r2[lens]
        xa = (dd * dd + a * a - b * b) / (2.0 * dd)      # centre 1 to the chord
        xb = dd - xa
        seg_a = a * a * np.arccos(np.clip(xa / a, -1.0, 1.0)) - xa * np.sqrt(np.maximum(a * a - xa * xa, 0.0))
        seg_b = b * b * np.arccos(np.clip(xb / b, -1.0, 1.0)) - xb * np.sqrt(np.maximum(b * b - xb * xb, 0.0))
        out[lens] = seg_a + seg_b
    return out


def disc_iou(x1, y1, r1, x2, y2, r2):
    """Intersection over union of two discs."""
    d = np.hypot(np.asarray(x1, np.float64) - x2, np.asarray(y1, np.float64) - y2)
    inter = disc_intersection(d, r1, r2)
    union = math.pi * (np.asarray(r1, np.float64) ** 2 + np.asarray(r2, np.float64) ** 2) - inter
    return inter / union


@dataclasses.dataclass
class Match:
    tp: int
    fp: int
    fn: int
    precision: float
    recall: float
    pairs: np.ndarray          # (tp, 2) detection index, ground-truth index


def match(det_xyr, scores, gt_xyr, iou: float = 0.5) -> Match:
    """Greedy VOC matching of detections (N, 3) with scores (N,) against
    ground-truth circles (M, 3); columns x, y, r."""
    det = np.asarray(det_xyr, np.float64).reshape(-1, 3)
    gt = np.asarray(gt_xyr, np.float64).reshape(-1, 3)
    n, m = det.shape[0], gt.shape[0]
    order = np.argsort(-np.asarray(scores, np.float64), kind="stable")
    taken = np.zeros(m, dtype=bool)
    pairs = []
    if n and m:
        # candidate pairs: discs that meet, found through a grid of cells at
        # least as wide as the largest pair of radii
        cell = max(1.0, 2.0 * (det[:, 2].max() + gt[:, 2].max()))
        gx = np.floor(gt[:, 0] / cell).astype(np.int64)
        gy = np.floor(gt[:, 1] / cell).astype(np.int64)
        buckets: dict = {}
        for j, key in enumerate(zip(gx.tolist(), gy.tolist())):
            buckets.setdefault(key, []).append(j)
        for i in order:
            x, y, r = det[i]
            cx, cy = int(math.floor(x / cell)), int(math.floor(y / cell))
            cand = [j for ox in (-1, 0, 1) for oy in (-1, 0, 1) for j in buckets.get((cx + ox, cy + oy), ())
                    if not taken[j]]
            if not cand:
                continue
            c = np.asarray(cand)
            v = disc_iou(x, y, r, gt[c, 0], gt[c, 1], gt[c, 2])
            k = int(np.argmax(v))
            if v[k] >= iou:
                taken[c[k]] = True
                pairs.append((int(i), int(c[k])))
    tp = len(pairs)
    fp = n - tp
    fn = m - tp
    return Match(tp, fp, fn, tp / n if n else 1.0, tp / m if m else 1.0,
                 np.asarray(pairs, dtype=np.int64).reshape(-1, 2))


def blob_circles(x, y, sigma):
    """(N, 3) circles of detected blobs: radius sqrt(2) sigma (Sec. 4)."""
    return np.stack([np.asarray(x, np.float64), np.asarray(y, np.float64),
                     math.sqrt(2.0) * np.asarray(sigma, np.float64)], axis=1)
