"""Pins of the oracle's DoG, maximum test and candidate list (Sec. 3, Eq. 1-3,
Sec. 4, Sec. 4.1) against scipy/torch library routines, the closed-form
response of an isolated Gaussian blob, and invariants."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

import oracle
from paper_2010_08486_gb300 import synth

CFG1 = oracle.OracleParams(min_sigma=1.0, max_sigma=10.0, ratio=1.6, threshold=0.1)
CFG2 = oracle.OracleParams(min_sigma=0.8, ratio=1.1, n_levels=25, threshold=0.05)


def test_ladders():
    s1 = oracle.ladder(CFG1)
    assert len(s1) == 6 and s1[-1] >= 10.0 and s1[-2] < 10.0
    np.testing.assert_allclose(s1, 1.6 ** np.arange(6), rtol=1e-15)
    s2 = oracle.ladder(CFG2)
    assert len(s2) == 25
    np.testing.assert_allclose(s2[-1], 0.8 * 1.1 ** 24, rtol=1e-15)
    assert list(oracle.radii(s1, 4.0)) == [4, 6, 10, 16, 26, 42]
    assert int(np.sum(2 * oracle.radii(s2, 4.0) + 1)) == 659
    # Eq. 1: arithmetic ladder of n_bin + 1 kernels from min to max.
    pa = oracle.OracleParams(min_sigma=1.0, max_sigma=5.0, n_levels=5, ladder=oracle.LADDER_ARITH)
    np.testing.assert_allclose(oracle.ladder(pa), [1, 2, 3, 4, 5], rtol=0, atol=1e-15)


def test_norm_coeffs_closed_forms():
    s = oracle.ladder(CFG2)
    np.testing.assert_allclose(oracle.norm_coeffs(s, oracle.NORM_DERIV), 1.0 / 0.1, rtol=1e-12)
    np.testing.assert_allclose(oracle.norm_coeffs(s, oracle.NORM_PAPER), s[:-1], rtol=0)


@pytest.mark.parametrize("norm", [oracle.NORM_DERIV, oracle.NORM_PAPER])
def test_dog_equals_scipy_composition(norm):
    img = synth.small_blob_frame(1, 64, 80, n_blobs=4).astype(np.float64)
    sig = oracle.ladder(CFG1)
    D = oracle.dog(img, sig, oracle.radii(sig, 4.0), norm)
    L = [ndi.gaussian_filter(img, s, mode="reflect", truncate=4.0) for s in sig]
    for i in range(len(sig) - 1):
        c = sig[i] if norm == oracle.NORM_PAPER else sig[i] / (sig[i + 1] - sig[i])
        np.testing.assert_allclose(D[i], c * (L[i] - L[i + 1]), rtol=0, atol=1e-13)


def _random_cube(seed, shape=(5, 17, 23)):
    rng = np.random.default_rng(seed)
    D = rng.normal(size=shape)
    # plateaus: quantise part of the cube so that ties occur
    D[1] = np.round(D[1] * 2) / 2
    D[3, :4, :4] = 0.7
    return D


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_local_max_equals_scipy_maximum_filter(seed):
    D = _random_cube(seed)
    thr = 0.1
    lyx, resp = oracle.local_max(D, thr)
    mx = ndi.maximum_filter(D, size=3, mode="constant", cval=-np.inf)
    want = np.argwhere((D == mx) & (D > thr))
    assert np.array_equal(lyx, want)
    np.testing.assert_array_equal(resp, D[tuple(want.T)])


@pytest.mark.parametrize("seed", [3, 4])
def test_local_max_equals_torch_max_pool3d(seed):
    D = _random_cube(seed, (4, 9, 31))
    t = torch.from_numpy(D)[None, None]
    mp = torch.nn.functional.max_pool3d(t, kernel_size=3, stride=1, padding=1)[0, 0].numpy()
    lyx, _ = oracle.local_max(D, 0.0)
    want = np.argwhere((mp - D == 0) & (D > 0.0))   # Sec. 4.1 Thresh definition
    assert np.array_equal(lyx, want)
    m = oracle.max_mask(D)
    assert np.array_equal(np.argwhere(m), np.argwhere(mp == D))


def test_threshold_is_strict():
    D = np.zeros((3, 5, 5))
    D[1, 2, 2] = 0.1
    assert len(oracle.local_max(D, 0.1)[0]) == 0
    D[1, 2, 2] = np.nextafter(0.1, 1.0)
    assert len(oracle.local_max(D, 0.1)[0]) == 1


def _isolated(ratio, levels, amp=0.8, spacing=None, n_levels=25, min_sigma=0.8):
    p = oracle.OracleParams(min_sigma=min_sigma, ratio=ratio, n_levels=n_levels, threshold=0.05,
                            prune=oracle.PRUNE_OFF)
    sig = oracle.ladder(p)
    R = int(oracle.radii(sig, 4.0).max())
    s_list = [sig[j] * math.sqrt(ratio) for j in levels]
    spacing = spacing or int(2 * R + 12 * max(s_list) + 8)
    n = len(levels)
    h, w = spacing, spacing * n
    centres = [(spacing // 2 + k * spacing, spacing // 2) for k in range(n)]
    img = np.zeros((h, w))
    for (cx, cy), s in zip(centres, s_list):
        img += synth.isolated_blob_frame(h, w, [(cx, cy)], s, amp)
    return p, sig, img, centres, s_list


def test_closed_form_blob_response_and_level_r11():
    # DERIV normalisation: the centre response peaks at sigma = s / sqrt(r)
    # with value A / (r + 1) (heat-equation argument of Sec. 3, Fig. 3).
    levels = [10, 13, 16]
    p, sig, img, centres, s_list = _isolated(1.1, levels)
    det = oracle.detect(img, p, keep_dog=True)
    keys = det.candidates.keys()
    for j, (cx, cy) in zip(levels, centres):
        assert (j, cy, cx) in keys
        d = det.D[j, cy, cx]
        assert abs(d - oracle.continuum_peak_response(0.8, 1.1)) < 1e-3 * 0.8 / 2.1
        assert int(np.argmax(det.D[:, cy, cx])) == j
    assert len(det.candidates) == len(levels)


def test_closed_form_blob_response_r16():
    p = oracle.OracleParams(min_sigma=1.0, ratio=1.6, n_levels=6, threshold=0.1, prune=oracle.PRUNE_OFF)
    sig = oracle.ladder(p)
    j = 2
    s = sig[j] * math.sqrt(1.6)
    n = 200
    img = synth.isolated_blob_frame(n, n, [(100, 100)], s, 1.0)
    det = oracle.detect(img, p, keep_dog=True)
    assert (j, 100, 100) in det.candidates.keys()
    assert abs(det.D[j, 100, 100] - 1.0 / 2.6) < 1e-3 / 2.6
    # the full centre curve follows the continuum closed form
    for i in range(len(sig) - 1):
        want = oracle.continuum_centre_response(1.0, s, sig[i], 1.6)
        assert abs(det.D[i, 100, 100] - want) < 2e-3 * want + 1e-4


def test_paper_normalisation_peak_location():
    # Eq. 3 literally (c_i = sigma_i) moves the peak to sigma ~ 1.653 s at r = 1.1.
    p = oracle.OracleParams(min_sigma=0.8, ratio=1.1, n_levels=25, norm=oracle.NORM_PAPER)
    sig = oracle.ladder(p)
    s = 2.5
    img = synth.isolated_blob_frame(161, 161, [(80, 80)], s, 1.0)
    D = oracle.dog(img, sig, oracle.radii(sig, 4.0), oracle.NORM_PAPER)
    j = int(np.argmax(D[:, 80, 80]))
    assert 1.653 / 1.1 <= sig[j] / s <= 1.653 * 1.1


def test_response_unimodal_in_scale():
    # Sec. 3 / Fig. 3: at a blob centre the response rises then falls with scale.
    p, sig, img, centres, _ = _isolated(1.1, [12])
    D = oracle.dog(img, sig, oracle.radii(sig, 4.0))
    cx, cy = centres[0]
    curve = D[:, cy, cx]
    k = int(np.argmax(curve))
    assert np.all(np.diff(curve[: k + 1]) > 0) and np.all(np.diff(curve[k:]) < 0)


def test_constant_image_gives_no_blobs():
    img = np.full((48, 40), 0.6)
    for p in (CFG1, CFG2):
        det = oracle.detect(img, p, keep_dog=True)
        assert np.max(np.abs(det.D)) < 1e-12
        assert len(det.candidates) == 0 and len(det.blobs) == 0


def test_affine_invariance():
    img = synth.small_blob_frame(5, 96, 96, n_blobs=6).astype(np.float64)
    sig = oracle.ladder(CFG1)
    rad = oracle.radii(sig, 4.0)
    D1 = oracle.dog(img, sig, rad)
    D2 = oracle.dog(2.5 * img + 0.3, sig, rad)
    np.testing.assert_allclose(D2, 2.5 * D1, rtol=0, atol=1e-12)


def test_transpose_and_flip_equivariance():
    img = synth.small_blob_frame(9, 100, 90, n_blobs=8).astype(np.float64)
    p = CFG1
    base = oracle.candidates(img, p)
    kt = oracle.candidates(img.T.copy(), p).keys()
    assert kt == {(l, x, y) for (l, y, x) in base.keys()}
    kf = oracle.candidates(img[:, ::-1].copy(), p).keys()
    assert kf == {(l, y, img.shape[1] - 1 - x) for (l, y, x) in base.keys()}
    kv = oracle.candidates(img[::-1, :].copy(), p).keys()
    assert kv == {(l, img.shape[0] - 1 - y, x) for (l, y, x) in base.keys()}


def test_small_frame_recovers_most_truth():
    # Sec. 4: radius r = sqrt(2) sigma.  Blobs of the 256x256 generator whose
    # size lies inside the ladder and that sit away from the border are found
    # near their true centre at a level whose sigma is within one ladder step.
    img, truth = synth.small_blob_frame(1, return_truth=True)
    det = oracle.detect(img.astype(np.float64), CFG1)
    sig = oracle.ladder(CFG1)
    found = 0
    considered = 0
    for cx, cy, s in zip(truth.cx, truth.cy, truth.s):
        if not (12 < cx < 244 and 12 < cy < 244) or s > sig[-2] * math.sqrt(1.6):
            continue
        considered += 1
        d = np.hypot(det.blobs.x - cx, det.blobs.y - cy)
        k = np.argmin(d)
        if d[k] <= 2.0 and 1 / 1.6 ** 1.5 <= det.blobs.sigma[k] * math.sqrt(1.6) / s <= 1.6 ** 1.5:
            found += 1
    assert considered >= 8
    assert found >= 0.7 * considered
