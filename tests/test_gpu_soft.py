"""Differentiable form on the GPU vs the FP64 oracle: soft histogram and its
gradient with respect to the frame and the sigma ladder.

The oracle is evaluated with the GPU's own local-maximum mask (computed from
the GPU's dumped responses with the same >= rule), so that the comparison
isolates the arithmetic; the mask itself is pinned by the detection tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import _lib, dog, synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def crop(seed, y0=480, x0=480, n=64):
    return synth.plif_frame(seed)[y0:y0 + n, x0:x0 + n].copy()


def setup(img, scale=1.0):
    cfg = dog.grad_config(max_h=img.shape[0], max_w=img.shape[1])
    det = dog.Detector(cfg)
    p = parity.oracle_params(cfg)
    sig0 = np.asarray(det.sigmas)
    # 0.1% perturbation: the radii floor(4 sigma + 0.5) of this ladder stay fixed
    sig = (sig0 * (1.0 + 0.001 * np.sin(np.arange(len(sig0))) * scale)).astype(np.float32)
    return cfg, det, p, sig0, sig


def gpu_mask(det, img_t, sig):
    # the mask at the perturbed sigmas: a detector built on that ladder dumps D
    cfg = dog.grad_config(sigmas=[float(s) for s in sig], max_h=img_t.shape[0], max_w=img_t.shape[1])
    cfg.sigmas = [float(s) for s in sig]
    d2 = dog.Detector(cfg)
    assert d2.radii == det.radii
    D = d2.debug_dog(img_t).cpu().numpy().astype(np.float64)
    return oracle.max_mask(D)


def record_mask(rec, shape):
    """The maxima the forward recorded, as a (P, H, W) mask; no duplicates."""
    n = int(rec.count)
    assert n <= rec.cap
    r = rec.buf[:n].cpu().numpy()
    x, y, l = r[:, 0], r[:, 1], r[:, 2]
    m = np.zeros(shape, dtype=bool)
    m[l, y, x] = True
    assert int(m.sum()) == n, "a maximum was recorded twice"
    return m


def check_record_mask(rec, img, sig, rad, p):
    """The recorded maxima equal the oracle's own 3x3x3 maxima (no threshold)
    of its FP64 responses at the same sigmas, except at voxels within 1e-4 of
    their largest neighbour (undecidable in FP32).  Returns the record mask."""
    D = oracle.dog(img.astype(np.float64), np.asarray(sig, np.float64), rad, p.norm)
    m_rec = record_mask(rec, D.shape)
    m_ora = oracle.max_mask(D)
    diff = m_rec ^ m_ora
    undecidable = np.abs(D - parity.max26(D)) <= parity.DECIDE
    assert not np.any(diff & ~undecidable), "decidable maxima differ at %d voxels" % int(np.sum(diff & ~undecidable))
    return m_rec


@pytest.mark.parametrize("n", [64, 200])
def test_soft_hist_matches_oracle(n):
    img = crop(synth.GRAD_SEED_BASE, n=n)
    cfg, det, p, sig0, sig = setup(img)
    t = torch.from_numpy(img).cuda()
    s = torch.from_numpy(sig).cuda()
    H = det.soft_hist(t, s).cpu().numpy().astype(np.float64)
    rad = np.asarray(det.radii)
    mask = gpu_mask(det, t, sig)
    Ho = oracle.soft_hist(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0, mask)
    assert np.abs(H - Ho).max() <= 1e-4 * Ho.sum() + 1e-5
    # accumulation semantics: a second call adds the same histogram again
    H2 = det.soft_hist(t, s, out=torch.from_numpy(H.astype(np.float32)).cuda()).cpu().numpy()
    np.testing.assert_allclose(H2, 2 * H, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("use_rec", [False, True])
@pytest.mark.parametrize("n", [64, 160])
def test_backward_matches_oracle_gradient(n, use_rec):
    img = crop(synth.GRAD_SEED_BASE, n=n)
    cfg, det, p, sig0, sig = setup(img)
    t = torch.from_numpy(img).cuda()
    s = torch.from_numpy(sig).cuda()
    rad = np.asarray(det.radii)
    tgt = oracle.soft_hist(crop(synth.GRAD_TARGET_SEED_BASE, n=n).astype(np.float64), sig0, rad, p, sig0)
    rec = None
    if use_rec:   # the forward's list of maxima instead of recomputing the blur levels
        rec = dog.SoftMaxima(1 << 16, "cuda")
        det.soft_hist(t, s, rec=rec)
        assert 0 < int(rec.count) <= rec.cap and det.status() == 0
        mask = check_record_mask(rec, img, sig, rad, p)
    else:
        mask = gpu_mask(det, t, sig)
    Ho = oracle.soft_hist(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0, mask)
    gH = 2.0 * (Ho - tgt)
    gi, gs = det.backward(t, s, torch.from_numpy(gH.astype(np.float32)).cuda(), rec=rec)
    gi, gs = gi.cpu().numpy().astype(np.float64), gs.cpu().numpy().astype(np.float64)
    oi, osg = oracle.soft_grad(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0,
                               gH.astype(np.float32).astype(np.float64), mask)
    assert np.linalg.norm(gi - oi) <= 1e-4 * np.linalg.norm(oi)
    assert np.linalg.norm(gs - osg) <= 1e-4 * np.linalg.norm(osg)


@pytest.mark.parametrize("shape", [(40, 1), (40, 7), (33, 30), (37, 31), (50, 61)])
def test_soft_narrow_frames_match_oracle(shape):
    """The soft modes run 32-column strips stepping by 30 from column -1:
    frames of one strip, of exactly 30 columns, of one column more, and of
    two strips give the oracle's soft histogram and record every maximum the
    oracle finds (decidable voxels), each once."""
    h, w = shape
    img = synth.plif_frame(synth.GRAD_SEED_BASE + 7)[500:500 + h, 600:600 + w].copy()
    cfg, det, p, sig0, sig = setup(img)
    t = torch.from_numpy(img).cuda()
    s = torch.from_numpy(sig).cuda()
    rad = np.asarray(det.radii)
    rec = dog.SoftMaxima(1 << 16, "cuda")
    H = det.soft_hist(t, s, rec=rec).cpu().numpy().astype(np.float64)
    assert det.status() == 0
    mask = check_record_mask(rec, img, sig, rad, p)
    Ho = oracle.soft_hist(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0, mask)
    assert np.abs(H - Ho).max() <= 1e-4 * Ho.sum() + 1e-5


@pytest.mark.parametrize("use_rec", [False, True])
def test_backward_odd_shape_matches_oracle(use_rec):
    # width not a multiple of 4 (no vectorised staging), height not a multiple
    # of the adjoint tiles, both wider than 2 R (one reflected copy per edge)
    img = synth.plif_frame(synth.GRAD_SEED_BASE + 5)[300:450, 400:573].copy()
    cfg, det, p, sig0, sig = setup(img)
    t = torch.from_numpy(img).cuda()
    s = torch.from_numpy(sig).cuda()
    rad = np.asarray(det.radii)
    mask = gpu_mask(det, t, sig)
    Ho = oracle.soft_hist(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0, mask)
    gH = (2.0 * (Ho - 0.5 * Ho.mean())).astype(np.float32)
    rec = None
    if use_rec:
        rec = dog.SoftMaxima(1 << 16, "cuda")
        det.soft_hist(t, s, rec=rec)
        assert 0 < int(rec.count) <= rec.cap and det.status() == 0
    gi, gs = det.backward(t, s, torch.from_numpy(gH).cuda(), rec=rec)
    assert det.status() == 0
    gi, gs = gi.cpu().numpy().astype(np.float64), gs.cpu().numpy().astype(np.float64)
    oi, osg = oracle.soft_grad(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0,
                               gH.astype(np.float64), mask)
    assert np.linalg.norm(gi - oi) <= 1e-4 * np.linalg.norm(oi)
    assert np.linalg.norm(gs - osg) <= 1e-4 * np.linalg.norm(osg)


def test_autograd_function_matches_backward():
    imgs = np.stack([crop(synth.GRAD_SEED_BASE + f, n=96) for f in range(3)])
    cfg, det, p, sig0, sig = setup(imgs[0])
    frames = torch.from_numpy(imgs).cuda().requires_grad_(True)
    sigmas = torch.from_numpy(sig).cuda().requires_grad_(True)
    target = torch.zeros(cfg.nbins, device="cuda")
    H = dog.DoGSoftHist.apply(frames, sigmas, det)
    loss = ((H - target) ** 2).sum()
    loss.backward()
    gH = (2 * (H - target)).detach()
    gs = torch.zeros(det.K, device="cuda")
    for b in range(3):
        # the autograd backward scatters from the forward's maxima; the plain
        # backward recomputes them: same gradient up to FP32 rounding order
        gi, _ = det.backward(frames[b].detach(), sigmas.detach(), gH, grad_sigmas=gs)
        assert torch.linalg.norm(frames.grad[b] - gi) <= 1e-5 * torch.linalg.norm(gi)
    # the record path evaluates the kernel-shape sigma term at the maxima only
    # (the recomputing path as dense inner products): same sum, other order
    assert torch.linalg.norm(sigmas.grad - gs) <= 1e-4 * torch.linalg.norm(gs)
    # the batch histogram is the sum of the per-frame histograms
    Hs = sum(det.soft_hist(frames[b].detach(), sigmas.detach()) for b in range(3))
    torch.testing.assert_close(H.detach(), Hs, rtol=1e-5, atol=1e-5)


def test_record_overflow_falls_back_to_recompute(monkeypatch):
    # an all-zero frame ties every voxel (D == 0, each one a >= maximum): the
    # record overflows, the status says so, and the autograd backward
    # recomputes that frame instead
    img = crop(synth.GRAD_SEED_BASE, n=64)
    cfg, det, p, sig0, sig = setup(img)
    flat = np.zeros_like(img)
    frames = torch.from_numpy(np.stack([img, flat])).cuda().requires_grad_(True)
    sigmas = torch.from_numpy(sig).cuda().requires_grad_(True)
    rec = dog.SoftMaxima(64, "cuda")
    det.soft_hist(frames[1].detach(), sigmas.detach(), rec=rec)
    assert int(rec.count) == (det.K - 1) * 64 * 64
    assert det.status() == _lib.DOG_ERR_CAPACITY
    assert det.status() == 0
    monkeypatch.setattr(dog.DoGSoftHist, "rec_cap", 4096)
    H = dog.DoGSoftHist.apply(frames, sigmas, det)
    (H ** 2).sum().backward()
    assert det.status() == 0
    gH = (2 * H).detach()
    gi, _ = det.backward(frames[1].detach(), sigmas.detach(), gH)
    torch.testing.assert_close(frames.grad[1], gi, rtol=0, atol=0)


def test_full_frame_gradient_matches_oracle():
    """A whole 1024x1024 frame of the differentiable workload (12 sigmas
    1.25^k, perturbed by 0.1%): the forward's record equals the oracle's own
    maxima on decidable voxels, and the gradients with respect to the frame
    and the sigmas match the oracle's analytic gradient (relative L2 1e-4),
    the oracle evaluated with the recorded maxima."""
    img = synth.plif_frame(synth.GRAD_SEED_BASE)
    cfg, det, p, sig0, sig = setup(img)
    t = torch.from_numpy(img).cuda()
    s = torch.from_numpy(sig).cuda()
    rad = np.asarray(det.radii)
    rec = dog.SoftMaxima(1 << 18, "cuda")
    H = det.soft_hist(t, s, rec=rec).cpu().numpy().astype(np.float64)
    assert det.status() == 0
    mask = check_record_mask(rec, img, sig, rad, p)
    Ho = oracle.soft_hist(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0, mask)
    assert np.abs(H - Ho).max() <= 1e-4 * Ho.sum() + 1e-5
    gH = (2.0 * (Ho - 0.5 * Ho.mean())).astype(np.float32)
    gi, gs = det.backward(t, s, torch.from_numpy(gH).cuda(), rec=rec)
    assert det.status() == 0
    gi, gs = gi.cpu().numpy().astype(np.float64), gs.cpu().numpy().astype(np.float64)
    oi, osg = oracle.soft_grad(img.astype(np.float64), sig.astype(np.float64), rad, p, sig0,
                               gH.astype(np.float64), mask)
    assert np.linalg.norm(gi - oi) <= 1e-4 * np.linalg.norm(oi)
    assert np.linalg.norm(gs - osg) <= 1e-4 * np.linalg.norm(osg)
