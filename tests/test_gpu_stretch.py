"""Contrast stretch on the GPU (Sec. 4, the optional preprocessing step: a
frame is stretched to [0, 1] with 0.35% saturation) against the FP64 oracle:
integer limits exactly, stretched values bit for bit, and detection with the
stretch fused into the 12-bit ingest equal to detection of the oracle's
stretched frame, single-frame and batched."""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth
from tests import parity

pytestmark = pytest.mark.gpu
SAT = 0.0035


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def counts_t(c):
    return torch.from_numpy(np.ascontiguousarray(c).view(np.int16)).cuda()


def frames():
    rng = np.random.default_rng(11)
    out = {
        "plif_1024": synth.plif_frame_u16(synth.PLIF_SEED_BASE, 1024, 1024),
        "plif_768x1024": synth.plif_frame_u16(synth.BATCH_SEED_BASE + 3, 768, 1024),
        "poisson_ties": rng.poisson(900, size=(256, 256)).astype(np.uint16),
        "odd_37x53": rng.integers(0, 4096, size=(37, 53)).astype(np.uint16),
        "row_1x1000": rng.integers(0, 4096, size=(1, 1000)).astype(np.uint16),
        "col_1000x1": rng.integers(0, 4096, size=(1000, 1)).astype(np.uint16),
        "tiny_3x3": np.arange(9, dtype=np.uint16).reshape(3, 3) * 400,
        "single": np.array([[77]], dtype=np.uint16),
        "constant": np.full((64, 64), 2048, dtype=np.uint16),
        "over_12bit": rng.integers(3000, 65535, size=(128, 96)).astype(np.uint16),
    }
    return out


@pytest.mark.parametrize("name", list(frames().keys()))
def test_limits_and_values_match_oracle(name):
    c = frames()[name]
    lo, hi = oracle.stretch_limits(c, SAT)
    lohi = dog.stretch_limits(counts_t(c), SAT)
    out = dog.stretch(counts_t(c), lohi)
    torch.cuda.synchronize()
    assert tuple(lohi.cpu().tolist()) == (lo, hi)
    want = oracle.stretch(c, lo, hi)
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), \
        "stretched values differ at %d pixels" % np.count_nonzero(got != want)


def test_pitched_frame():
    base = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 1, 300, 512)
    t = counts_t(base)[:, 3:403]             # pitch 512, width 400
    c = base[:, 3:403]
    assert tuple(dog.stretch_limits(t, SAT).cpu().tolist()) == oracle.stretch_limits(c, SAT)
    assert np.array_equal(dog.stretch(t, sat=SAT).cpu().numpy(), oracle.preprocess(c, SAT))


def test_saturation_fractions():
    for sat in (0.0, 0.01, 0.2):
        c = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 2, 256, 256)
        assert tuple(dog.stretch_limits(counts_t(c), sat).cpu().tolist()) == oracle.stretch_limits(c, sat)


def test_fused_ingest_equals_detection_of_stretched_frame():
    """Detection of the 12-bit frame with the stretch fused into the ingest is
    bit-identical to detection of the oracle's stretched FP32 frame."""
    c = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 3, 512, 512)
    pre = oracle.preprocess(c, SAT)
    det_s = dog.Detector(dog.plif_config(stretch_sat=SAT, max_h=512, max_w=512, blob_cap=16384))
    det = dog.Detector(dog.plif_config(max_h=512, max_w=512, blob_cap=16384))
    D_s = det_s.debug_dog(counts_t(c)).cpu().numpy()
    D = det.debug_dog(torch.from_numpy(pre).cuda()).cpu().numpy()
    assert np.array_equal(D_s, D)
    b_s, h_s, _ = det_s.detect(counts_t(c))
    b, h, _ = det.detect(torch.from_numpy(pre).cuda())
    torch.cuda.synchronize()
    assert parity.same_blob_sets(parity.blobs_to_oracle(*b_s.to_numpy()), parity.blobs_to_oracle(*b.to_numpy()))
    assert np.array_equal(h_s.cpu().numpy(), h.cpu().numpy())
    assert det_s.status() == 0


def test_stretched_detection_matches_oracle():
    """D of the stretched 12-bit frame within the parity tolerance of the
    oracle's D of its own stretched frame; decidable candidates identical;
    pruning and histogram equal to the oracle's on the GPU candidates."""
    c = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 4, 384, 448)
    cfg = dog.plif_config(stretch_sat=SAT, max_h=384, max_w=448, blob_cap=16384)
    det = dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    pre = oracle.preprocess(c, SAT).astype(np.float64)
    sig = oracle.ladder(p)
    rad = oracle.radii(sig, p.truncate)
    D_ora = oracle.dog(pre, sig, rad, p.norm)
    D_gpu = det.debug_dog(counts_t(c)).cpu().numpy()
    parity.check_dog_values(D_gpu, D_ora, oracle.norm_coeffs(sig, p.norm), 1.0)
    cand = det.candidates(counts_t(c))
    torch.cuda.synchronize()
    x, y, l, s, r = cand.to_numpy()
    parity.compare_candidates(set(zip(l.tolist(), y.tolist(), x.tolist())), D_ora, cfg.threshold)
    pr = det.prune(cand, 384, 448)
    hist, _ = det.volume_hist(pr)
    torch.cuda.synchronize()
    ora_pr = oracle.prune(parity.blobs_to_oracle(x, y, l, s, r), p)
    ora_pr.sigma = ora_pr.sigma.astype(np.float32).astype(np.float64)
    gpu_pr = parity.blobs_to_oracle(*pr.to_numpy())
    assert parity.same_blob_sets(gpu_pr, ora_pr)
    assert np.array_equal(hist.cpu().numpy(), oracle.hist(gpu_pr, p)[0].astype(np.int32))


def test_batched_stretch_equals_per_frame():
    """A mixed batch (12-bit frames stretched, FP32 frames used as given) in one
    persistent launch equals the single-frame calls."""
    shapes = [(128, 128), (256, 512), (37, 61), (512, 512), (200, 96)]
    imgs = []
    for f, (h, w) in enumerate(shapes):
        if f % 2 == 0:
            imgs.append(counts_t(synth.plif_frame_u16(synth.BATCH_SEED_BASE + 20 + f, h, w)))
        else:
            imgs.append(torch.from_numpy(synth.plif_frame(synth.BATCH_SEED_BASE + 20 + f, h, w)).cuda())
    cap = 8192
    det = dog.Detector(dog.plif_config(stretch_sat=SAT, max_h=512, max_w=512, blob_cap=cap))
    want = []
    for img in imgs:
        b, h, _ = det.detect(img)
        torch.cuda.synchronize()
        x, y, l, s, r = b.to_numpy()
        want.append((sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist(), r.tolist())), h.cpu().numpy()))
    table = det.frame_table(imgs, cap)
    n = len(imgs)
    out = torch.empty((n * cap, 5), dtype=torch.int32, device="cuda")
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    hists = torch.zeros((n, det.nbins_out), dtype=torch.int32, device="cuda")
    for _ in range(2):   # the batch workspace keeps the last call's contents
        det.detect_batched(None, table=table, out=out, counts=counts, hists=hists)
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        for f in range(n):
            x, y, l, s, r = dog.blobs_from_raw(out[f * cap:(f + 1) * cap], int(c[f]))
            got = sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist(), r.tolist()))
            assert got == want[f][0], "frame %d" % f
            assert np.array_equal(hists[f].cpu().numpy(), want[f][1])
    assert det.status() == 0
