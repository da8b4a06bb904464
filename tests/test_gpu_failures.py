"""Failure handling without a GPU fault: allocation failures injected on the
host (dog_test_fail_alloc) make dog_create and the batched workspace growth
return DOG_ERR_NOMEM, free what they had allocated, and leave the handle (or
the library) usable; a capacity overflow reports the true count."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2010_08486_gb300 import _lib
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()
    yield
    _lib.load().dog_test_fail_alloc(-1)


def _create(cfg):
    lib = _lib.load()
    c, keep = cfg.to_c()
    h = ctypes.c_void_p()
    st = lib.dog_create(ctypes.byref(c), ctypes.byref(h))
    return st, h


def test_create_fails_cleanly_at_every_allocation():
    lib = _lib.load()
    cfg = dog.plif_config(max_h=512, max_w=512, blob_cap=4096)
    st, h = _create(cfg)          # warm-up: context and module state
    assert st == _lib.DOG_OK
    lib.dog_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    hit = 0
    for k in range(64):
        lib.dog_test_fail_alloc(k)
        st, h = _create(cfg)
        lib.dog_test_fail_alloc(-1)
        if st == _lib.DOG_OK:      # fewer than k + 1 allocations: nothing failed
            lib.dog_destroy(h)
            break
        assert st == _lib.DOG_ERR_NOMEM, "allocation %d: %s" % (k, st)
        assert h.value is None
        hit += 1
    assert hit >= 10, "dog_create made only %d workspace allocations" % hit
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (4 << 20), "device memory leaked"


def test_batch_growth_failure_then_recovery():
    lib = _lib.load()
    shapes = [(256, 256), (128, 320), (200, 96)]
    imgs = [torch.from_numpy(synth.plif_frame(synth.BATCH_SEED_BASE + 60 + f, h, w)).cuda()
            for f, (h, w) in enumerate(shapes)]
    det = dog.Detector(dog.plif_config(max_h=320, max_w=320, blob_cap=4096))
    lib.dog_test_fail_alloc(3)
    with pytest.raises(_lib.DogError) as e:
        det.detect_batched(imgs)
    lib.dog_test_fail_alloc(-1)
    assert e.value.code == _lib.DOG_ERR_NOMEM
    # the next call grows the workspace again and gives the per-frame results
    out, counts, hists = det.detect_batched(imgs)
    torch.cuda.synchronize()
    cap = det.cfg.blob_cap
    for f, img in enumerate(imgs):
        b, h, _ = det.detect(img)
        torch.cuda.synchronize()
        x, y, l, s, r = b.to_numpy()
        want = sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist()))
        x2, y2, l2, s2, r2 = dog.blobs_from_raw(out[f * cap:(f + 1) * cap], int(counts[f]))
        assert sorted(zip(l2.tolist(), y2.tolist(), x2.tolist(), s2.tolist())) == want
        assert np.array_equal(hists[f].cpu().numpy(), h.cpu().numpy())
    assert det.status() == 0


def test_capacity_overflow_keeps_handle_usable():
    img = torch.from_numpy(synth.plif_frame(synth.PLIF_SEED_BASE, 256, 256)).cuda()
    det = dog.Detector(dog.plif_config(max_h=256, max_w=256, blob_cap=8192))
    small = dog.empty_blobs(16, "cuda")
    det.candidates(img, out=small)
    torch.cuda.synchronize()
    full = det.candidates(img)
    torch.cuda.synchronize()
    assert small.n() == full.n() > 16            # the true count is reported
    assert det.status() == _lib.DOG_ERR_CAPACITY
    assert det.status() == 0                     # reading clears it
    again = det.candidates(img)
    torch.cuda.synchronize()
    assert again.n() == full.n() and det.status() == 0
