"""CUDA path vs FP64 oracle: DoG responses, candidates, pruning, histogram
(Sec. 3-4 / Sec. 4.1), through the C ABI on the GPU."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth
from paper_2010_08486_gb300 import _lib
from tests import parity

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_candidates(det, img_t):
    c = det.candidates(img_t)
    torch.cuda.synchronize()
    x, y, l, s, r = c.to_numpy()
    return c, (x, y, l, s, r)


def full_check(cfg, img_np, det=None, img_t=None, check_prune=True):
    """D values, candidate sets, prune and histogram of one frame."""
    det = det or dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    img32 = img_np.astype(np.float32) if img_np.dtype != np.uint16 else synth.u16_to_f32(img_np)
    img_t = img_t if img_t is not None else dev(img32)
    sig = oracle.ladder(p)
    np.testing.assert_allclose(det.sigmas, sig, rtol=1e-15, atol=0)
    assert det.radii == list(oracle.radii(sig, p.truncate))
    D_ora = oracle.dog(img32.astype(np.float64), sig, oracle.radii(sig, p.truncate), p.norm)
    c = oracle.norm_coeffs(sig, p.norm)
    D_gpu = det.debug_dog(img_t).cpu().numpy()
    parity.check_dog_values(D_gpu, D_ora, c, float(np.abs(img32).max()))
    cand, (x, y, l, s, r) = gpu_candidates(det, img_t)
    keys = set(zip(l.tolist(), y.tolist(), x.tolist()))
    assert len(keys) == len(x), "duplicate candidates"
    n_undecided = parity.compare_candidates(keys, D_ora, cfg.threshold)
    # responses are the dumped D values, sigma the plane sigma
    np.testing.assert_array_equal(r, D_gpu[l, y, x])
    np.testing.assert_array_equal(s, np.asarray(sig, np.float32)[l])
    if not check_prune:
        return det, n_undecided
    H, W = img32.shape
    pr = det.prune(cand, H, W)
    hist, vol = det.volume_hist(pr, with_volume=True)
    torch.cuda.synchronize()
    gpu_pr = parity.blobs_to_oracle(*pr.to_numpy())
    ora_pr = oracle.prune(parity.blobs_to_oracle(x, y, l, s, r), p)
    ora_pr.sigma = ora_pr.sigma.astype(np.float32).astype(np.float64)
    assert parity.same_blob_sets(gpu_pr, ora_pr), "prune differs"
    counts, vols = oracle.hist(gpu_pr, p)
    np.testing.assert_array_equal(hist.cpu().numpy(), counts.astype(np.int32))
    np.testing.assert_allclose(vol.cpu().numpy(), vols, rtol=1e-12, atol=0)
    # composite entry point gives the same blobs and histogram
    blobs, h2, _ = det.detect(img_t)
    torch.cuda.synchronize()
    assert parity.same_blob_sets(parity.blobs_to_oracle(*blobs.to_numpy()), gpu_pr)
    np.testing.assert_array_equal(h2.cpu().numpy(), hist.cpu().numpy())
    assert det.status() == 0
    return det, n_undecided


def test_small_frame_matches_oracle():
    cfg = dog.small_frame_config()
    img = synth.small_blob_frame(1)
    _, und = full_check(cfg, img)
    assert und == 0


def test_small_frame_matches_stored_fixture():
    with open(os.path.join(HERE, "golden", "small_frame_seed1.json")) as f:
        gold = json.load(f)
    det = dog.Detector(dog.small_frame_config())
    blobs, hist, _ = det.detect(dev(synth.small_blob_frame(1)))
    torch.cuda.synchronize()
    x, y, l, s, r = blobs.to_numpy()
    got = sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist()))
    assert got == sorted(tuple(b[:4]) for b in gold["blobs"])
    assert hist.cpu().tolist() == gold["counts"]


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (37, 1), (5, 3), (9, 40), (33, 65), (70, 31),
                                   (100, 129), (64, 96)])
def test_odd_shapes_match_oracle(shape):
    h, w = shape
    rng = np.random.default_rng(h * 1000 + w)
    img = np.clip(0.4 + 0.2 * rng.standard_normal((h, w)), 0, 1)
    if h > 8 and w > 8:
        img += synth.isolated_blob_frame(h, w, [(w // 2, h // 2), (w // 3, h // 4)], 2.2, 0.8)
    cfg = dog.small_frame_config(threshold=0.02, max_h=max(h, 8), max_w=max(w, 8))
    full_check(cfg, img.astype(np.float32))


def test_constant_and_zero_frames_have_no_blobs():
    det = dog.Detector(dog.plif_config(max_h=128, max_w=160))
    for v in (0.0, 0.37, 1.0):
        img = dev(np.full((128, 160), v, np.float32))
        blobs, hist, _ = det.detect(img)
        torch.cuda.synchronize()
        assert blobs.n() == 0 and int(hist.sum()) == 0
        D = det.debug_dog(img).cpu().numpy()
        assert np.abs(D).max() < 1e-5


def test_blobs_on_strip_edges():
    # centres on both sides of the 32-column strip boundaries exercise the
    # queued-and-resolved path for neighbours held by another strip
    h, w = 96, 160
    centres = [(31, 20), (32, 50), (63, 80), (64, 30), (95, 60), (96, 15), (127, 75), (128, 45)]
    img = 0.1 + synth.isolated_blob_frame(h, w, centres, 2.0, 0.9)
    cfg = dog.small_frame_config(threshold=0.05, max_h=h, max_w=w)
    det, und = full_check(cfg, img.astype(np.float32))
    cand, (x, y, l, s, r) = gpu_candidates(det, dev(img.astype(np.float32)))
    found = set(zip(x.tolist(), y.tolist()))
    for c in centres:
        assert c in found


def test_u16_ingest_matches_f32():
    counts = synth.plif_frame_u16(synth.PLIF_SEED_BASE, 200, 230)
    cfg = dog.plif_config(max_h=200, max_w=230)
    det = dog.Detector(cfg)
    t16 = dev(counts.view(np.int16))
    t32 = dev(synth.u16_to_f32(counts))
    D16 = det.debug_dog(t16).cpu().numpy()
    D32 = det.debug_dog(t32).cpu().numpy()
    assert np.array_equal(D16, D32)
    a = det.candidates(t16).to_numpy()
    b = det.candidates(t32).to_numpy()
    assert sorted(zip(a[2], a[1], a[0])) == sorted(zip(b[2], b[1], b[0]))
    full_check(cfg, counts, det=det, img_t=t16)


def test_u16_pitched_and_offset_frames_match_f32():
    """A 12-bit frame given contiguously, with a pitch of 2 mod 4 counts and a
    base offset by one count, or padded to a pitch of 324, single and
    batched, gives the f32 path's D and candidates exactly."""
    counts = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 3, 256, 320)
    cfg = dog.plif_config(max_h=256, max_w=320)
    det = dog.Detector(cfg)
    want_D = det.debug_dog(dev(synth.u16_to_f32(counts))).cpu().numpy()
    want_c = sorted(zip(*det.candidates(dev(synth.u16_to_f32(counts))).to_numpy()))
    wide = np.zeros((256, 326), np.uint16)
    wide[:, 1:321] = counts
    wide_t = dev(wide.view(np.int16))
    views = {"contiguous": dev(counts.view(np.int16)),
             "pitch_326": wide_t[:, 1:321],                 # pitch 2 mod 4, base 2 bytes off
             "pitch_324": dev(np.pad(counts, ((0, 0), (0, 4))).view(np.int16))[:, :320]}
    for name, t in views.items():
        assert np.array_equal(det.debug_dog(t).cpu().numpy(), want_D), name
        assert sorted(zip(*det.candidates(t).to_numpy())) == want_c, name
    _, cnt, hist = det.detect_batched(list(views.values()))
    b, h, _ = det.detect(views["contiguous"])
    torch.cuda.synchronize()
    assert cnt.cpu().tolist() == [b.n()] * 3
    for f in range(3):
        assert np.array_equal(hist[f].cpu().numpy(), h.cpu().numpy())


def test_row_bands_match_whole_frame():
    img = synth.plif_frame(synth.PLIF_SEED_BASE + 7, 300, 200)
    det = dog.Detector(dog.plif_config(max_h=300, max_w=200))
    t = dev(img)
    D0 = det.debug_dog(t).cpu().numpy()
    k0 = sorted(zip(*det.candidates(t).to_numpy()[:3]))
    for band in (8, 64, 136):
        det.set_tiling(band)
        assert np.array_equal(det.debug_dog(t).cpu().numpy(), D0)
        assert sorted(zip(*det.candidates(t).to_numpy()[:3])) == k0
    det.set_tiling(0)


@pytest.mark.parametrize("ladder", ["plif", "grad"])
def test_kernel_forms_agree_bit_for_bit(ladder):
    """The 8- and 12-producer-warp forms compute every level with the same
    operations: D, candidates and the pruned blobs are identical, single frame
    and batched, whichever form the handle picked by default."""
    cfg = (dog.plif_config if ladder == "plif" else dog.grad_config)(max_h=300, max_w=200)
    img = synth.plif_frame(synth.PLIF_SEED_BASE + 11, 300, 200)
    det = dog.Detector(cfg)
    assert det.producer_warps == (12 if ladder == "plif" else 8)
    t = dev(img)
    out = {}
    for nw in (8, 12):
        det.set_producer_warps(nw)
        assert det.producer_warps == nw
        D = det.debug_dog(t).cpu().numpy()
        cand = sorted(zip(*det.candidates(t).to_numpy()))
        b, h, _ = det.detect(t)
        bb, cc, hh = det.detect_batched([t, t[:150, :120].contiguous()])
        torch.cuda.synchronize()
        out[nw] = (D, cand, sorted(zip(*b.to_numpy())), h.cpu().numpy(), cc.cpu().numpy(), hh.cpu().numpy())
    assert np.array_equal(out[8][0], out[12][0])
    for a, b in zip(out[8][1:], out[12][1:]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    det.set_producer_warps(0)
    assert det.producer_warps == (12 if ladder == "plif" else 8)
    with pytest.raises(_lib.DogError) as e:
        det.set_producer_warps(10)
    assert e.value.code == _lib.DOG_ERR_INVALID


def test_capacity_overflow_reports_true_count():
    det = dog.Detector(dog.small_frame_config())
    img = dev(synth.small_blob_frame(1))
    full = det.candidates(img).n()
    assert full > 5
    c = det.candidates(img, cap=5)
    assert c.n() == full
    assert det.status() == _lib.DOG_ERR_CAPACITY
    assert det.status() == 0


def test_plif_full_size_matches_oracle():
    # the benchmark's frame size and ladder: 1024x1024 12-bit, 25 levels 0.8 * 1.1^i
    counts = synth.plif_frame_u16(synth.PLIF_SEED_BASE)
    cfg = dog.plif_config()
    det = dog.Detector(cfg)
    _, und = full_check(cfg, counts, det=det, img_t=dev(counts.view(np.int16)))
    assert und <= 5


def test_paper_normalisation_and_arithmetic_ladder():
    img = synth.small_blob_frame(4, 120, 140, n_blobs=8)
    cfg = dog.DetectorConfig(min_sigma=1.0, max_sigma=6.0, n_levels=8, ladder=_lib.LADDER_ARITH,
                             norm=_lib.NORM_PAPER, threshold=0.05, max_h=120, max_w=140)
    full_check(cfg, img)


@pytest.mark.parametrize("mode", [_lib.PRUNE_SUPPRESS, _lib.PRUNE_OFF])
def test_prune_modes(mode):
    cfg = dog.plif_config(prune=mode, max_h=256, max_w=256)
    full_check(cfg, synth.plif_frame(synth.PLIF_SEED_BASE + 3, 256, 256))


def test_ladder_histogram_mode():
    cfg = dog.plif_config(hist_mode=_lib.HIST_LADDER, max_h=256, max_w=256)
    full_check(cfg, synth.plif_frame(synth.PLIF_SEED_BASE + 4, 256, 256))


def test_explicit_sigma_ladder():
    sig = [0.9, 1.3, 1.7, 2.6, 3.1, 4.4, 6.0]
    cfg = dog.DetectorConfig(sigmas=sig, threshold=0.05, max_h=150, max_w=150)
    full_check(cfg, synth.plif_frame(synth.PLIF_SEED_BASE + 5, 150, 150))


def test_detect_recovers_isolated_blobs_at_known_radius():
    # closed form: a Gaussian blob of std s = sigma_j sqrt(r) peaks on plane j with
    # response A / (r + 1), so its radius sqrt(2) sigma_j is recovered
    cfg = dog.plif_config(max_h=256, max_w=512, threshold=0.05)
    det = dog.Detector(cfg)
    levels = [8, 12, 16]
    centres = [(90, 128), (256, 128), (420, 128)]
    img = np.zeros((256, 512))
    for j, c in zip(levels, centres):
        img += synth.isolated_blob_frame(256, 512, [c], det.sigmas[j] * np.sqrt(1.1), 0.8)
    blobs, hist, _ = det.detect(dev(img.astype(np.float32)))
    torch.cuda.synchronize()
    x, y, l, s, r = blobs.to_numpy()
    got = {(int(a), int(b)): (int(c), float(d), float(e)) for a, b, c, d, e in zip(x, y, l, s, r)}
    for j, c in zip(levels, centres):
        lev, sg, resp = got[c]
        assert lev == j and sg == np.float32(det.sigmas[j])
        assert abs(resp - 0.8 / 2.1) < 1e-3 * 0.8 / 2.1


def test_prune_many_candidates_global_path():
    """More candidates than the pruning kernel copies to shared memory (4096):
    it then works on the global arrays; the result is the oracle's prune of the
    same candidate list."""
    cfg = dog.plif_config(threshold=0.0, max_h=512, max_w=512)
    img = synth.plif_frame(synth.PLIF_SEED_BASE + 7, 512, 512)
    det = dog.Detector(cfg)
    cand, (x, y, l, s, r) = gpu_candidates(det, dev(img))
    assert len(x) > 4096
    pr = det.prune(cand, 512, 512)
    torch.cuda.synchronize()
    p = parity.oracle_params(cfg)
    gpu_pr = parity.blobs_to_oracle(*pr.to_numpy())
    ora_pr = oracle.prune(parity.blobs_to_oracle(x, y, l, s, r), p)
    ora_pr.sigma = ora_pr.sigma.astype(np.float32).astype(np.float64)
    assert parity.same_blob_sets(gpu_pr, ora_pr), "prune differs"
    assert det.status() == 0
