"""dog_prune_noalloc: pruning for callers that may not allocate device memory
(for example a plug-in whose host framework owns all device memory and
forbids allocations inside its execution step).  It must return what
dog_prune returns for the same candidates, on consecutive calls that reuse
its fixed internal scratch array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2010_08486_gb300 import _lib
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth

pytestmark = pytest.mark.gpu


def _blob_set(raw, n):
    r = raw[:n].cpu()
    f = r[:, 3:].view(torch.float32)
    return sorted(zip(r[:, 2].tolist(), r[:, 1].tolist(), r[:, 0].tolist(), f[:, 0].tolist(), f[:, 1].tolist()))


@pytest.mark.parametrize("prune", [_lib.PRUNE_COALESCE, _lib.PRUNE_SUPPRESS])
def test_noalloc_prune_equals_handle_prune_twice(prune):
    libbuild.build()
    lib = _lib.load()
    cfg = dog.plif_config(prune=prune, max_h=512, max_w=512, blob_cap=16384)
    det = dog.Detector(cfg)
    sig = (ctypes.c_double * det.P)(*det.sigmas[:det.P])
    for seed in (11, 12):
        img = torch.from_numpy(synth.plif_frame(synth.PLIF_SEED_BASE + seed, 512, 512)).cuda()
        cand = det.candidates(img)
        want = det.prune(cand, 512, 512)
        torch.cuda.synchronize()
        n_want = want.n()
        assert n_want > 100
        for _ in range(2):   # two calls in a row share the scratch array
            out = torch.full((16384, 5), -1, dtype=torch.int32, device="cuda")
            nout = torch.zeros((), dtype=torch.int32, device="cuda")
            st = lib.dog_prune_noalloc(cand.raw.data_ptr(), cand.count.data_ptr(), cand.raw.shape[0], sig, det.P,
                                       cfg.overlap, prune, out.data_ptr(), out.shape[0], nout.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
            assert st == _lib.DOG_OK
            torch.cuda.synchronize()
            assert int(nout) == n_want
            assert _blob_set(out, n_want) == _blob_set(want.raw, n_want)


def test_noalloc_rejects_oversized_input():
    libbuild.build()
    lib = _lib.load()
    sig = (ctypes.c_double * 3)(1.0, 1.6, 2.56)
    buf = torch.zeros((4, 5), dtype=torch.int32, device="cuda")
    cnt = torch.zeros((), dtype=torch.int32, device="cuda")
    st = lib.dog_prune_noalloc(buf.data_ptr(), cnt.data_ptr(), _lib.NOALLOC_MAX_CAND + 1, sig, 3, 0.5,
                               _lib.PRUNE_COALESCE, buf.data_ptr(), 4, cnt.data_ptr(), None)
    assert st == _lib.DOG_ERR_UNSUPPORTED
