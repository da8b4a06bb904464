"""FFT-convolution backend (Sec. 4.1's alternative to direct convolution)
against the FP64 oracle and the direct path.

The FFTs run in single precision, so D carries the transforms' rounding
(which scales with the frame's norm rather than with each sample); measured,
it stays below 4% of the direct path's tolerance, so the FFT backend is held
to the same rule: |D - D_oracle| <= 1e-5 * c_i * max|I| per voxel, and the
candidate sets must match the oracle's on every voxel decidable at the 1e-4
margin.  Prints the worst error of each case in units of that tolerance."""
import json

import numpy as np
import pytest
import torch

import oracle
from paper_2010_08486_gb300 import _lib
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth
from tests import parity

pytestmark = pytest.mark.gpu
FFT_D_RTOL = parity.D_RTOL


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _check(cfg, img32, u16=None, name=""):
    det = dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    sig = oracle.ladder(p)
    rad = oracle.radii(sig, p.truncate)
    c = oracle.norm_coeffs(sig, p.norm)
    img_t = torch.from_numpy(u16.view(np.int16) if u16 is not None else img32).cuda()
    D_ora = oracle.dog(img32.astype(np.float64), sig, rad, p.norm)
    D_fft = det.debug_dog(img_t).cpu().numpy()
    amax = max(float(np.abs(img32).max()), 1e-30)
    err = np.abs(D_fft.astype(np.float64) - D_ora) / (np.asarray(c)[:, None, None] * amax)
    print(json.dumps({"case": name, "shape": list(img32.shape), "levels": len(sig),
                      "worst_err_over_direct_tol": float(err.max() / parity.D_RTOL),
                      "rms_err_over_direct_tol": float(np.sqrt((err ** 2).mean()) / parity.D_RTOL)}))
    assert err.max() <= FFT_D_RTOL
    cand = det.candidates(img_t)
    torch.cuda.synchronize()
    x, y, l, s, r = cand.to_numpy()
    keys = set(zip(l.tolist(), y.tolist(), x.tolist()))
    assert len(keys) == len(x)
    parity.compare_candidates(keys, D_ora, cfg.threshold)
    np.testing.assert_array_equal(r, D_fft[l, y, x])
    # detect = candidates -> coalescing -> histogram, as the oracle on them
    b, hist, _ = det.detect(img_t)
    torch.cuda.synchronize()
    ora = oracle.prune(parity.blobs_to_oracle(x, y, l, s, r), p)
    ora.sigma = ora.sigma.astype(np.float32).astype(np.float64)
    got = parity.blobs_to_oracle(*b.to_numpy())
    assert parity.same_blob_sets(got, ora)
    assert np.array_equal(hist.cpu().numpy(), oracle.hist(got, p)[0].astype(np.int32))
    assert det.status() == 0
    return det


def test_fft_plif_full_frame():
    u16 = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 7)
    _check(dog.plif_config(backend=_lib.BACKEND_FFT), synth.u16_to_f32(u16), u16, "plif_1024_u16")


def test_fft_small_frame_workload():
    img = synth.small_blob_frame(1)
    _check(dog.small_frame_config(backend=_lib.BACKEND_FFT), img, name="small_256")


@pytest.mark.parametrize("shape", [(37, 61), (9, 300), (128, 7)])
def test_fft_odd_and_folded_frames(shape):
    # radii up to 42 on frames narrower than the kernels: repeated reflection
    h, w = shape
    img = synth.small_blob_frame(5, h, w, n_blobs=4)
    _check(dog.small_frame_config(backend=_lib.BACKEND_FFT, max_h=h, max_w=w), img, name="odd_%dx%d" % shape)


def test_fft_with_contrast_stretch_and_smaller_frames():
    cfg = dog.plif_config(backend=_lib.BACKEND_FFT, stretch_sat=0.0035, max_h=512, max_w=512)
    u16 = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 8, 512, 512)
    det = _check(cfg, oracle.preprocess(u16, 0.0035), u16, "plif_512_stretched")
    # a smaller frame after a larger one on the same workspace
    u16b = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 9, 300, 200)
    D = det.debug_dog(torch.from_numpy(u16b.view(np.int16)).cuda()).cpu().numpy()
    p = parity.oracle_params(cfg)
    sig = oracle.ladder(p)
    D_ora = oracle.dog(oracle.preprocess(u16b, 0.0035).astype(np.float64), sig, oracle.radii(sig, 4.0), p.norm)
    c = oracle.norm_coeffs(sig, p.norm)
    assert (np.abs(D - D_ora) / np.asarray(c)[:, None, None]).max() <= FFT_D_RTOL


def test_fft_batched_is_unsupported():
    det = dog.Detector(dog.plif_config(backend=_lib.BACKEND_FFT, max_h=64, max_w=64))
    img = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.DogError) as e:
        det.detect_batched([img])
    assert e.value.code == _lib.DOG_ERR_UNSUPPORTED


def test_fft_ladder_beyond_direct_shared_memory():
    """25 levels up to sigma 14 (radii to 56) do not fit the fused kernel's
    shared memory; the FFT backend still builds and matches the oracle, while
    the direct backend reports UNSUPPORTED."""
    ratio = (14.0 / 0.8) ** (1.0 / 24)
    with pytest.raises(_lib.DogError) as e:
        dog.Detector(dog.plif_config(ratio=ratio, max_h=384, max_w=384))
    assert e.value.code == _lib.DOG_ERR_UNSUPPORTED
    cfg = dog.plif_config(ratio=ratio, backend=_lib.BACKEND_FFT, max_h=384, max_w=384)
    u16 = synth.plif_frame_u16(synth.PLIF_SEED_BASE + 10, 384, 384)
    det = _check(cfg, synth.u16_to_f32(u16), u16, "plif_384_sigma14")
    sig = torch.ones(det.K, dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.DogError) as e2:
        det.soft_hist(torch.zeros((384, 384), dtype=torch.float32, device="cuda"), sig)
    assert e2.value.code == _lib.DOG_ERR_UNSUPPORTED
