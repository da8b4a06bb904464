"""Seeded synthetic frames for the DoG blob detector.

This module only draws inputs; it holds none of the detector's arithmetic, and
both the CUDA path and the FP64 oracle are fed from it.  The paper evaluates
on frames rendered from 100 spheres plus Poisson and Gaussian noise at
1000x1000 (Sec. 5) and on real PLIF frames (Sec. 2); neither is available, so
isotropic Gaussian blobs at integer pixel centres stand in for droplets:

    blob(x, y) = A * exp(-((x - cx)^2 + (y - cy)^2) / (2 s^2)),

evaluated exactly inside the square window |x - cx| <= 6 s, |y - cy| <= 6 s.

Every generator takes an integer seed and uses numpy's PCG64, so a frame is a
pure function of (recipe, seed, size).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

U16_FULL_SCALE = 4095  # 12-bit PLIF camera range


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _add_blobs(img: np.ndarray, cx, cy, s, amp) -> None:
    """Add Gaussian blobs to ``img`` (float64, H x W) in place."""
    h, w = img.shape
    for x0, y0, sd, a in zip(cx, cy, s, amp):
        half = 6.0 * sd
        xlo = max(0, int(math.ceil(x0 - half)))
        xhi = min(w - 1, int(math.floor(x0 + half)))
        ylo = max(0, int(math.ceil(y0 - half)))
        yhi = min(h - 1, int(math.floor(y0 + half)))
        if xlo > xhi or ylo > yhi:
            continue
        xs = np.arange(xlo, xhi + 1, dtype=np.float64) - x0
        ys = np.arange(ylo, yhi + 1, dtype=np.float64) - y0
        gx = np.exp(-(xs * xs) / (2.0 * sd * sd))
        gy = np.exp(-(ys * ys) / (2.0 * sd * sd))
        img[ylo:yhi + 1, xlo:xhi + 1] += a * np.outer(gy, gx)


@dataclasses.dataclass(frozen=True)
class BlobTruth:
    """Ground-truth blob parameters of a generated frame (pixel units)."""
    cx: np.ndarray
    cy: np.ndarray
    s: np.ndarray
    amp: np.ndarray


def small_blob_frame(seed: int = 1, h: int = 256, w: int = 256, n_blobs: int = 20,
                     return_truth: bool = False):
    """256x256 FP32 frame: 20 blobs, s ~ U[1, 8], A ~ U[0.3, 1], N(0, 0.02) noise.

    Positions are uniform on [0, w) x [0, h); the result is clipped to [0, 1].
    """
    rng = _rng(seed)
    cx = rng.uniform(0.0, float(w), n_blobs)
    cy = rng.uniform(0.0, float(h), n_blobs)
    s = rng.uniform(1.0, 8.0, n_blobs)
    amp = rng.uniform(0.3, 1.0, n_blobs)
    img = np.zeros((h, w), dtype=np.float64)
    _add_blobs(img, cx, cy, s, amp)
    img += rng.normal(0.0, 0.02, size=(h, w))
    out = np.clip(img, 0.0, 1.0).astype(np.float32)
    if return_truth:
        return out, BlobTruth(cx, cy, s, amp)
    return out


def plif_blob_count(h: int, w: int) -> int:
    """2000 blobs per 1024x1024 frame, scaled by area."""
    return int(round(2000.0 * h * w / (1024.0 * 1024.0)))


def plif_frame_u16(seed: int, h: int = 1024, w: int = 1024, n_blobs: int | None = None,
                   return_truth: bool = False):
    """PLIF-shaped 12-bit frame as uint16 counts in [0, 4095].

    Blobs: s = exp(N(ln 3, 0.5)) clipped to [0.8, 20], A ~ U[0.3, 1], centres
    uniform.  Background: a plume 0.25 * exp(-(x-w/2)^2/(2*120^2)
    - (y-h/2)^2/(2*300^2)) whose long axis is vertical.  The clean image is
    clipped to [0, 1]; counts = min(Poisson(4095 * clean), 4095).
    """
    rng = _rng(seed)
    n = plif_blob_count(h, w) if n_blobs is None else int(n_blobs)
    cx = rng.uniform(0.0, float(w), n)
    cy = rng.uniform(0.0, float(h), n)
    s = np.clip(np.exp(rng.normal(math.log(3.0), 0.5, n)), 0.8, 20.0)
    amp = rng.uniform(0.3, 1.0, n)
    xs = np.arange(w, dtype=np.float64) - w / 2.0
    ys = np.arange(h, dtype=np.float64) - h / 2.0
    img = 0.25 * np.outer(np.exp(-(ys * ys) / (2.0 * 300.0 ** 2)),
                          np.exp(-(xs * xs) / (2.0 * 120.0 ** 2)))
    _add_blobs(img, cx, cy, s, amp)
    clean = np.clip(img, 0.0, 1.0)
    counts = np.minimum(rng.poisson(U16_FULL_SCALE * clean), U16_FULL_SCALE).astype(np.uint16)
    if return_truth:
        return counts, BlobTruth(cx, cy, s, amp)
    return counts


def u16_to_f32(counts: np.ndarray) -> np.ndarray:
    """12-bit counts to FP32 in [0, 1]: one IEEE single division by 4095 per pixel."""
    return counts.astype(np.float32) / np.float32(U16_FULL_SCALE)


def plif_frame(seed: int, h: int = 1024, w: int = 1024) -> np.ndarray:
    """FP32 PLIF-shaped frame in [0, 1]."""
    return u16_to_f32(plif_frame_u16(seed, h, w))


PLIF_SEED_BASE = 2_000_000
BATCH_SEED_BASE = 3_000_000
GRAD_SEED_BASE = 4_000_000
GRAD_TARGET_SEED_BASE = 4_001_000
SERVE_SEED_BASE = 5_000

BATCH_SIZES = ((128, 128), (256, 512), (512, 512), (768, 1024), (1024, 1280))


def batch_shapes(n_frames: int = 256, seed: int = BATCH_SEED_BASE):
    """Uneven (h, w) shapes drawn uniformly from BATCH_SIZES with a seeded choice."""
    rng = _rng(seed)
    idx = rng.integers(0, len(BATCH_SIZES), size=n_frames)
    return [BATCH_SIZES[i] for i in idx]


def batch_frames(n_frames: int = 256, seed: int = BATCH_SEED_BASE):
    """Uneven-size FP32 PLIF-shaped frames, frame f drawn from seed + 1 + f."""
    return [plif_frame(seed + 1 + f, h, w) for f, (h, w) in enumerate(batch_shapes(n_frames, seed))]


def isolated_blob_frame(h: int, w: int, centres, s, amp) -> np.ndarray:
    """Noise-free FP64 frame of blobs at the given integer centres (no clipping)."""
    img = np.zeros((h, w), dtype=np.float64)
    cx = [c[0] for c in centres]
    cy = [c[1] for c in centres]
    _add_blobs(img, cx, cy, np.broadcast_to(np.asarray(s, dtype=np.float64), (len(cx),)),
               np.broadcast_to(np.asarray(amp, dtype=np.float64), (len(cx),)))
    return img


SPHERE_SEED_BASE = 6_000_000


def sphere_table(seed: int, n: int = 100, h: int = 1000, w: int = 1000, r_range=(3.0, 20.0),
                 amp_range=(0.3, 1.0)) -> np.ndarray:
    """(n, 4) float32 sphere table (cx, cy, R, A) for the rendered-sphere frames
    of the paper's evaluation (100 spheres on 1000 x 1000 frames): centres
    uniform over the frame, radii uniform in r_range (pixels), brightness
    uniform in amp_range."""
    g = _rng(seed)
    cx = g.uniform(0, w, n)
    cy = g.uniform(0, h, n)
    r = g.uniform(r_range[0], r_range[1], n)
    a = g.uniform(amp_range[0], amp_range[1], n)
    return np.stack([cx, cy, r, a], axis=1).astype(np.float32)
