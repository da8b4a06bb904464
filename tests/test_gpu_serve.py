"""Serving loop: frames from 8 camera streams of three sizes arrive as Poisson
processes; each result served in the continuous-batching mix equals the same
frame detected alone, and each stream's device-resident rolling histogram
equals the sum of its last `window` frame histograms."""
import numpy as np
import pytest
import torch

from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    libbuild.build()
    per_shape = {}
    for s, shape in enumerate(serve.SERVE_SHAPES):
        if shape not in per_shape:
            per_shape[shape] = [torch.from_numpy(synth.plif_frame_u16(synth.SERVE_SEED_BASE + 100 * len(per_shape) + k,
                                                                      *shape).view(np.int16)).pin_memory()
                                for k in range(3)]
    return [per_shape[shape] for shape in serve.SERVE_SHAPES]


def alone(det, frame):
    blobs, hist, _ = det.detect(frame.cuda())
    torch.cuda.synchronize()
    x, y, l, s, r = blobs.to_numpy()
    return sorted(zip(l.tolist(), y.tolist(), x.tolist(), s.tolist())), hist.cpu().numpy()


@pytest.mark.parametrize("max_batch,window", [(64, 250), (5, 7)])
def test_served_results_equal_alone(pool, max_batch, window):
    cfg = dog.plif_config(blob_cap=8192)
    srv = serve.StreamServer(cfg, serve.SERVE_SHAPES, window=window, mem_budget=256 << 20,
                             max_batch=max_batch, max_inflight=2, keep_blobs=True)
    sched = serve.poisson_schedule(len(serve.SERVE_SHAPES), 250.0, 0.25, 3, synth.SERVE_SEED_BASE)
    stats = srv.run(sched, pool)
    assert stats["frames"] == len(sched) == len(srv.finished)
    ref = {}
    det = dog.Detector(dog.plif_config(blob_cap=8192, max_h=1024, max_w=1280))
    for r in srv.finished:
        key = (r.sid, r.pool_idx)
        if key not in ref:
            ref[key] = alone(det, pool[r.sid][r.pool_idx])
        want_blobs, want_hist = ref[key]
        np.testing.assert_array_equal(r.hist, want_hist)
        assert r.count == len(want_blobs)
        raw = torch.from_numpy(r.blobs)
        got = sorted(zip(raw[:, 2].tolist(), raw[:, 1].tolist(), raw[:, 0].tolist(),
                         raw[:, 3:4].view(torch.float32)[:, 0].tolist()))
        assert got == want_blobs
    # rolling per-stream histograms: sum of each stream's last `window` frames
    sums = srv.rolling_hist()
    for s in range(len(serve.SERVE_SHAPES)):
        mine = sorted((r for r in srv.finished if r.sid == s), key=lambda r: r.t_arrival)
        want = np.sum([r.hist for r in mine[-window:]], axis=0) if mine else 0
        np.testing.assert_array_equal(sums[s], want)
    assert stats["p99_ms"] > 0 and stats["mp_per_s"] > 0
