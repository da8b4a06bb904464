"""Detection quality, GPU against the FP64 oracle (Sec. 5 reports that the
GPU and CPU detectors reach the same precision and recall on synthetic frames,
differences of order 1e-3): PASCAL-VOC matching (disc IoU >= 0.5) of each
detector's blobs against the generator's ground truth, on PLIF-shaped frames
(truth: circles of radius sqrt(2) s) and on rendered-sphere frames of the
paper's kind (100 spheres, 1000 x 1000, contrast stretched with 0.35%
saturation; truth: the spheres' discs).  Prints one JSON line per workload."""
import json

import numpy as np
import pytest
import torch

import oracle
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, quality, synth
from tests import parity

pytestmark = pytest.mark.gpu
TOL = 0.01    # |P_gpu - P_oracle| and |R_gpu - R_oracle| per frame


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _pr(x, y, sigma, resp, gt):
    m = quality.match(quality.blob_circles(x, y, sigma), resp, gt)
    return m.precision, m.recall


def _compare(name, det, p, frames):
    rows = []
    for counts, gt, ingest in frames:
        b, _, _ = det.detect(torch.from_numpy(counts.view(np.int16)).cuda())
        torch.cuda.synchronize()
        x, y, l, s, r = b.to_numpy()
        pg, rg = _pr(x, y, s, r, gt)
        ref = oracle.detect(ingest(counts).astype(np.float64), p)
        po, ro = _pr(ref.blobs.x, ref.blobs.y, ref.blobs.sigma, ref.blobs.response, gt)
        rows.append((pg, rg, po, ro))
    a = np.asarray(rows)
    dp, dr = a[:, 0] - a[:, 2], a[:, 1] - a[:, 3]
    print(json.dumps({"workload": name, "frames": len(rows), "precision_gpu": a[:, 0].mean(),
                      "recall_gpu": a[:, 1].mean(), "precision_oracle": a[:, 2].mean(),
                      "recall_oracle": a[:, 3].mean(), "dP_mean": dp.mean(), "dP_sd": dp.std(),
                      "dR_mean": dr.mean(), "dR_sd": dr.std()}))
    assert np.all(np.abs(dp) <= TOL) and np.all(np.abs(dr) <= TOL)
    return a


def test_precision_recall_plif_frames():
    cfg = dog.plif_config(max_h=512, max_w=512, blob_cap=16384)
    det = dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    frames = []
    for f in range(3):
        counts, truth = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 100 + f, 512, 512, return_truth=True)
        gt = np.stack([truth.cx, truth.cy, np.sqrt(2.0) * truth.s], axis=1)
        frames.append((counts, gt, synth.u16_to_f32))
    a = _compare("plif_512x512_u16", det, p, frames)
    assert a[:, 1].mean() > 0.3


def test_precision_recall_rendered_spheres():
    # ladder sigma = 2 * 1.15^i, 14 levels: DoG planes r = sqrt(2) sigma from 2.8 to 15 px
    cfg = dog.DetectorConfig(min_sigma=2.0, ratio=1.15, n_levels=14, threshold=0.05, max_h=1000, max_w=1000,
                             blob_cap=16384, stretch_sat=0.0035)
    det = dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    frames = []
    for f in range(2):
        seed = synth.SPHERE_SEED_BASE + 200 + f
        table = synth.sphere_table(seed, n=100, h=1000, w=1000, r_range=(4.0, 16.0))
        counts = dog.render_spheres(torch.from_numpy(table).cuda(), 1000, 1000, seed=seed)
        torch.cuda.synchronize()
        c = counts.cpu().numpy().view(np.uint16)
        frames.append((c, table[:, :3].astype(np.float64), lambda cc: oracle.preprocess(cc, 0.0035)))
    a = _compare("spheres_1000x1000_100", det, p, frames)
    assert a[:, 1].mean() > 0.5
