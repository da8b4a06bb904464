"""Parity rules between the CUDA path and the FP64 oracle.

Responses: |D_gpu - D_oracle| <= 1e-5 * c_i * max|I| per voxel (FP32 blur
error ~1e-6 relative, amplified by the normalisation c_i).  A candidate voxel
is decidable when its oracle response is more than 1e-4 away from the
threshold and from the largest of its in-range 26 neighbours; decidable
candidate sets must match exactly, undecidable ones may differ.  Pruning and
histogram are compared exactly on the GPU's own candidate list.
"""
import numpy as np

import oracle

D_RTOL = 1e-5
DECIDE = 1e-4


def oracle_params(cfg) -> oracle.OracleParams:
    """Oracle parameters from a DetectorConfig (field by field, no shared code)."""
    return oracle.OracleParams(min_sigma=cfg.min_sigma, max_sigma=cfg.max_sigma, ratio=cfg.ratio,
                               n_levels=cfg.n_levels, ladder=cfg.ladder,
                               sigmas=None if cfg.sigmas is None else tuple(cfg.sigmas),
                               truncate=cfg.truncate, threshold=cfg.threshold, overlap=cfg.overlap,
                               norm=cfg.norm, prune=cfg.prune, nbins=cfg.nbins, hist_mode=cfg.hist_mode,
                               soft_T=cfg.soft_T)


def max26(D):
    """Largest in-range 26-neighbour of every voxel (-inf where none)."""
    P, h, w = D.shape
    pad = np.full((P + 2, h + 2, w + 2), -np.inf)
    pad[1:-1, 1:-1, 1:-1] = D
    m = np.full(D.shape, -np.inf)
    for dl in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dl == dy == dx == 0:
                    continue
                m = np.maximum(m, pad[1 + dl:1 + dl + P, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w])
    return m


def check_dog_values(D_gpu, D_ora, c, img_absmax):
    tol = D_RTOL * np.asarray(c)[:, None, None] * max(img_absmax, 1e-30)
    err = np.abs(D_gpu.astype(np.float64) - D_ora)
    bad = err > tol
    assert not bad.any(), "D mismatch at %d voxels, worst %.3g vs tol %.3g" % (
        bad.sum(), err.max(), tol.max())
    return float((err / tol).max())


def compare_candidates(gpu_keys, D_ora, thr):
    """gpu_keys: set of (level, y, x).  Returns (n_decidable_mismatch, n_undecidable)."""
    lyx, _ = oracle.local_max(D_ora, thr)
    ora_keys = set(map(tuple, lyx.tolist()))
    m = max26(D_ora)
    diff = gpu_keys ^ ora_keys
    bad = []
    for (l, y, x) in diff:
        d = D_ora[l, y, x]
        if abs(d - thr) > DECIDE and abs(d - m[l, y, x]) > DECIDE:
            bad.append((l, y, x))
    assert not bad, "decidable candidates differ: %s" % bad[:10]
    return len(diff)


def blobs_to_oracle(x, y, level, sigma, resp):
    return oracle.Blobs(np.asarray(x, np.int32), np.asarray(y, np.int32), np.asarray(level, np.int32),
                        np.asarray(sigma, np.float64), np.asarray(resp, np.float64))


def same_blob_sets(a: oracle.Blobs, b: oracle.Blobs, check_sigma=True):
    ka = sorted(zip(a.level.tolist(), a.y.tolist(), a.x.tolist(),
                    np.asarray(a.sigma, np.float32).tolist() if check_sigma else [0] * len(a)))
    kb = sorted(zip(b.level.tolist(), b.y.tolist(), b.x.tolist(),
                    np.asarray(b.sigma, np.float32).tolist() if check_sigma else [0] * len(b)))
    return ka == kb
