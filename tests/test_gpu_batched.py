"""Batched detection of uneven frames in one persistent launch equals the
per-frame path, also with row bands and when replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth

pytestmark = pytest.mark.gpu

SIZES = [(128, 128), (256, 512), (37, 61), (512, 512), (768, 1024), (1024, 1280), (200, 96)]


@pytest.fixture(scope="module")
def frames():
    libbuild.build()
    return [torch.from_numpy(synth.plif_frame(synth.BATCH_SEED_BASE + 1 + f, h, w)).cuda()
            for f, (h, w) in enumerate(SIZES)]


def per_frame(det, frames):
    res = []
    for img in frames:
        blobs, hist, _ = det.detect(img)
        torch.cuda.synchronize()
        x, y, l, s, r = blobs.to_numpy()
        res.append((sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist(), r.tolist())),
                    hist.cpu().numpy()))
    return res


def unpack(det, out, counts, hists, n):
    cap = det.cfg.blob_cap
    c = counts.cpu().numpy()
    res = []
    for f in range(n):
        x, y, l, s, r = dog.blobs_from_raw(out[f * cap:(f + 1) * cap], int(c[f]))
        res.append((sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist(), r.tolist())),
                    hists[f].cpu().numpy()))
    return res


def assert_same(a, b):
    assert len(a) == len(b)
    for (ba, ha), (bb, hb) in zip(a, b):
        assert ba == bb
        np.testing.assert_array_equal(ha, hb)


def test_batched_equals_per_frame(frames):
    det = dog.Detector(dog.plif_config(max_h=1024, max_w=1280, blob_cap=8192))
    want = per_frame(det, frames)
    out, counts, hists = det.detect_batched(frames)
    torch.cuda.synchronize()
    assert_same(unpack(det, out, counts, hists, len(frames)), want)
    assert det.status() == 0
    # the persistent work counter resets itself: a second launch gives the same
    out, counts, hists = det.detect_batched(frames)
    torch.cuda.synchronize()
    assert_same(unpack(det, out, counts, hists, len(frames)), want)


def test_batched_varying_batch_sizes_on_one_handle(frames):
    # consecutive batched calls of different sizes reuse the handle's workspace
    det = dog.Detector(dog.plif_config(max_h=1024, max_w=1280, blob_cap=8192))
    want = per_frame(det, frames)
    for sel in ([0, 1, 2, 3, 4, 5, 6], [2], [5, 0], [1, 3, 6, 4], [6]):
        fr = [frames[i] for i in sel]
        out, counts, hists = det.detect_batched(fr)
        torch.cuda.synchronize()
        assert_same(unpack(det, out, counts, hists, len(fr)), [want[i] for i in sel])


@pytest.mark.parametrize("band,ctas", [(64, 1), (256, 1), (128, 2)])
def test_batched_row_bands(frames, band, ctas):
    det = dog.Detector(dog.plif_config(max_h=1024, max_w=1280, blob_cap=8192))
    want = per_frame(det, frames)
    det.set_tiling(band, ctas)
    out, counts, hists = det.detect_batched(frames)
    torch.cuda.synchronize()
    assert_same(unpack(det, out, counts, hists, len(frames)), want)


def test_batched_graph_replay(frames):
    det = dog.Detector(dog.plif_config(max_h=1024, max_w=1280, blob_cap=8192))
    want = per_frame(det, frames)
    table = det.frame_table(frames)
    n = len(frames)
    cap = det.cfg.blob_cap
    out = torch.empty((n * cap, 5), dtype=torch.int32, device="cuda")
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    hists = torch.zeros((n, det.nbins_out), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        det.detect_batched(None, table=table, out=out, counts=counts, hists=hists, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        det.detect_batched(None, table=table, out=out, counts=counts, hists=hists, stream=s)
    for _ in range(3):
        out.fill_(-1)
        counts.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert_same(unpack(det, out, counts, hists, n), want)


def test_autotuned_tiling_keeps_results(frames, tmp_path):
    from paper_2010_08486_gb300 import autotune
    det = dog.Detector(dog.plif_config(max_h=1024, max_w=1280, blob_cap=8192))
    want = per_frame(det, frames)
    table = det.frame_table(frames)
    res = autotune.tune_detector_batch(det, table, [tuple(f.shape) for f in frames],
                                       cache_path=str(tmp_path / "tune.json"))
    assert res.band % 8 == 0 and res.ms > 0 and len(res.timings) >= 2
    out, counts, hists = det.detect_batched(None, table=table)
    torch.cuda.synchronize()
    assert_same(unpack(det, out, counts, hists, len(frames)), want)
    # single-frame tuning on the largest frame
    r1 = autotune.tune_detector_frame(det, frames[5])
    blobs, hist, _ = det.detect(frames[5])
    torch.cuda.synchronize()
    x, y, l, s, r = blobs.to_numpy()
    assert sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist(), r.tolist())) == want[5][0]
    assert r1.band % 8 == 0
    assert det.status() == 0


def test_bench_launch_configuration_matches_per_frame_and_oracle_histogram():
    """The benchmark's launch: 96 uint16 1024x1024 frames in one persistent
    launch (the last round of tiles cut into finer bands).  Sampled frames give
    the blobs of the single-frame path, and histograms equal to the oracle's
    histogram of those blobs."""
    import oracle
    from tests import parity
    libbuild.build()
    distinct = [synth.plif_frame_u16(synth.PLIF_SEED_BASE + k) for k in range(12)]
    B = 96
    frames = torch.from_numpy(np.stack([distinct[f % 12].view(np.int16) for f in range(B)])).cuda()
    cfg = dog.plif_config(blob_cap=16384)
    det = dog.Detector(cfg)
    fl = [frames[f] for f in range(B)]
    out, counts, hists = det.detect_batched(fl)
    torch.cuda.synchronize()
    assert det.status() == 0
    got = unpack(det, out, counts, hists, B)
    p = parity.oracle_params(cfg)
    for f in (0, 47, 95):
        blobs, hist, _ = det.detect(fl[f])
        torch.cuda.synchronize()
        x, y, l, s, r = blobs.to_numpy()
        assert got[f][0] == sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist(), r.tolist()))
        np.testing.assert_array_equal(got[f][1], hist.cpu().numpy())
        want_counts, _ = oracle.hist(parity.blobs_to_oracle(x, y, l, s, r), p)
        np.testing.assert_array_equal(got[f][1], want_counts.astype(np.int32))


def test_batched_workload_sizes_match_oracle():
    """The batched and serving frame sizes checked against the FP64 oracle,
    not only against the per-frame GPU path: one persistent launch over a
    1024x1280, a 768x1024 and a 512x512 12-bit PLIF frame; per frame, the
    decidable candidates of the same frame equal the oracle's (Sec. 4.1
    threshold and 3x3x3 maximum), the batched pruned blobs equal the oracle's
    coalescing of those candidates, and the histogram equals the oracle's."""
    import oracle
    from tests import parity
    shapes = [(1024, 1280), (768, 1024), (512, 512)]
    counts_np = [synth.plif_frame_u16(synth.BATCH_SEED_BASE + 40 + f, h, w) for f, (h, w) in enumerate(shapes)]
    imgs = [torch.from_numpy(c.view(np.int16)).cuda() for c in counts_np]
    cap = 16384
    cfg = dog.plif_config(max_h=1024, max_w=1280, blob_cap=cap)
    det = dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    sig = oracle.ladder(p)
    rad = oracle.radii(sig, p.truncate)
    out, counts, hists = det.detect_batched(imgs)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    for f, (h, w) in enumerate(shapes):
        img32 = synth.u16_to_f32(counts_np[f])
        D_ora = oracle.dog(img32.astype(np.float64), sig, rad, p.norm)
        cand = det.candidates(imgs[f])
        torch.cuda.synchronize()
        x, y, l, s, r = cand.to_numpy()
        parity.compare_candidates(set(zip(l.tolist(), y.tolist(), x.tolist())), D_ora, cfg.threshold)
        ora_pr = oracle.prune(parity.blobs_to_oracle(x, y, l, s, r), p)
        ora_pr.sigma = ora_pr.sigma.astype(np.float32).astype(np.float64)
        got = parity.blobs_to_oracle(*dog.blobs_from_raw(out[f * cap:(f + 1) * cap], int(c[f])))
        assert parity.same_blob_sets(got, ora_pr), "frame %dx%d: batched blobs differ from the oracle" % (h, w)
        np.testing.assert_array_equal(hists[f].cpu().numpy(), oracle.hist(got, p)[0].astype(np.int32))
    assert det.status() == 0
