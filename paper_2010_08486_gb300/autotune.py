"""Tile-shape autotuner for the fused DoG detection kernel.

A tile of the fused kernel is a strip of 32 output columns by a band of rows.
Before its first output row a tile runs the horizontal passes of the rows its
vertical blur reaches above the band (the warm-up, about 8 * ceil((2 r_max +
1) / 8) rows), so a short band pays that halo often; a tall band leaves SMs
idle in the last wave (few tiles, one CTA per SM).  The best height depends on
the frame shapes, the ladder and the number of SMs, so it is measured.

The tuner ranks candidate band heights with a cost model (waves x rows walked,
the halo counted as half a row because only its horizontal pass runs), times
the best few on the device through the detector's own entry points, and keeps
the winner per (shapes, ladder) key.  It also times both kernel forms (8 or 12
producer warps; which is faster depends on the ladder).  The timing function
is injectable, so the selection logic runs on the CPU in tests.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

MB = 8          # rows per block of the fused kernel (band heights are multiples of it)
TX = 32         # columns per strip


def warmup_rows(radii: Sequence[int]) -> int:
    """Rows above a band whose horizontal pass a tile runs before its first
    output block: MB * max over levels of ceil((2 r + 1) / MB)."""
    return MB * max((2 * r + 1 + MB - 1) // MB for r in radii)


def tiles_of(shape: Tuple[int, int], band: int) -> int:
    h, w = shape
    nb = 1 if band <= 0 or band >= h else -(-h // band)
    return -(-w // TX) * nb


def model_cost(shapes: Sequence[Tuple[int, int]], band: int, radii: Sequence[int], n_sm: int,
               ctas_per_sm: int = 1) -> float:
    """Relative run time of one launch over `shapes` with row bands of `band`
    (0: whole frames): tiles are handed out in order to n_sm * ctas_per_sm
    persistent CTAs; each tile costs its rows + half its warm-up rows + 2 (the
    test's halo).  Greedy list scheduling of the tiles gives the makespan."""
    warm = warmup_rows(radii)
    slots = max(1, n_sm * ctas_per_sm)
    costs: List[float] = []
    for (h, w) in shapes:
        bh = h if band <= 0 or band >= h else band
        nb = -(-h // bh)
        ns = -(-w // TX)
        for b in range(nb):
            rows = min(bh, h - b * bh)
            costs.extend([rows + 2 + 0.5 * warm] * ns)
    if not costs:
        return 0.0
    if len(costs) > 64 * slots:
        # many tiles per CTA: the greedy makespan is within one tile of this
        return sum(costs) / slots + max(costs)
    # tiles are claimed in order by whichever CTA is free first
    import heapq
    heap = [0.0] * min(slots, len(costs))
    heapq.heapify(heap)
    for c in costs:
        t = heapq.heappop(heap)
        heapq.heappush(heap, t + c)
    return max(heap)


def candidate_bands(shapes: Sequence[Tuple[int, int]], radii: Sequence[int], n_sm: int,
                    ctas_per_sm: int = 1, limit: int = 4) -> List[int]:
    """Band heights worth timing, best modelled first.  0 (whole frames) is
    always among them."""
    hmax = max(h for h, _ in shapes)
    cands = {0}
    b = MB
    while b < hmax:
        cands.add(b)
        b += MB if b < 512 else 4 * MB
    ranked = sorted(cands, key=lambda c: (model_cost(shapes, c, radii, n_sm, ctas_per_sm), -c))
    out = ranked[:limit]
    if 0 not in out:
        out.append(0)
    return out


PRODUCER_WARPS = (12, 8)   # kernel forms (0: the handle's default)


@dataclass
class TuneResult:
    band: int
    ctas_per_sm: int
    ms: float
    timings: Dict[str, float] = field(default_factory=dict)
    producer_warps: int = 0


def shapes_key(shapes: Iterable[Tuple[int, int]], radii: Sequence[int], n_sm: int, mode: str) -> str:
    hist: Dict[Tuple[int, int], int] = {}
    for s in shapes:
        hist[tuple(s)] = hist.get(tuple(s), 0) + 1
    sh = ",".join("%dx%d*%d" % (h, w, n) for (h, w), n in sorted(hist.items()))
    return "%s|%s|r=%s|sm=%d" % (mode, sh, "-".join(map(str, radii)), n_sm)


class Autotuner:
    """Chooses band heights (and CTAs per SM) for a Detector by timing.

    measure(band, ctas_per_sm, producer_warps) -> milliseconds is supplied by
    the caller or built by `frame_measure` / `batch_measure`; results are
    cached per key and can be saved to / loaded from a JSON file."""

    def __init__(self, n_sm: int, radii: Sequence[int], cache_path: Optional[str] = None):
        self.n_sm = n_sm
        self.radii = list(radii)
        self.cache_path = cache_path
        self.cache: Dict[str, TuneResult] = {}
        if cache_path and os.path.exists(cache_path):
            self.load(cache_path)

    def tune(self, shapes: Sequence[Tuple[int, int]], measure: Callable[[int, int, int], float],
             mode: str = "frame", ctas_options: Sequence[int] = (1,), limit: int = 4,
             nw_options: Sequence[int] = PRODUCER_WARPS) -> TuneResult:
        key = shapes_key(shapes, self.radii, self.n_sm, mode)
        if key in self.cache:
            return self.cache[key]
        best: Optional[TuneResult] = None
        timings: Dict[str, float] = {}
        for nw in nw_options:
            for cps in ctas_options:
                for band in candidate_bands(shapes, self.radii, self.n_sm, cps, limit):
                    ms = float(measure(band, cps, nw))
                    timings["%d/%d/%d" % (band, cps, nw)] = ms
                    if not math.isfinite(ms):
                        continue
                    if best is None or ms < best.ms:
                        best = TuneResult(band, cps, ms, producer_warps=nw)
        if best is None:
            raise RuntimeError("autotune: no candidate tiling could be timed")
        best.timings = timings
        self.cache[key] = best
        if self.cache_path:
            self.save(self.cache_path)
        return best

    def save(self, path: str):
        with open(path, "w") as f:
            json.dump({k: vars(v) for k, v in self.cache.items()}, f, indent=1, sort_keys=True)

    def load(self, path: str):
        with open(path) as f:
            raw = json.load(f)
        for k, v in raw.items():
            self.cache[k] = TuneResult(int(v["band"]), int(v["ctas_per_sm"]), float(v["ms"]),
                                       {str(a): float(b) for a, b in v.get("timings", {}).items()},
                                       int(v.get("producer_warps", 0)))


def _time_ms(fn, reps: int, warm: int = 2) -> float:
    import torch
    for _ in range(warm):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _measure_with(det, fn, reps: int) -> Callable[[int, int, int], float]:
    def measure(band: int, cps: int, nw: int = 0) -> float:
        nw0 = det.producer_warps
        det.set_producer_warps(nw)
        det.set_tiling(band, cps)
        try:
            return _time_ms(fn, reps)
        finally:
            det.set_tiling(0, 1)
            det.set_producer_warps(nw0)
    return measure


def frame_measure(det, frame, reps: int = 5) -> Callable[[int, int, int], float]:
    """Timing function for single-frame detection (dog_detect) of `frame`."""
    import torch
    from . import dog
    blobs = dog.empty_blobs(det.cfg.blob_cap, frame.device)
    hist = torch.zeros(det.nbins_out, dtype=torch.int32, device=frame.device)
    return _measure_with(det, lambda: det.detect(frame, out=blobs, hist=hist), reps)


def batch_measure(det, table, reps: int = 3, **kw) -> Callable[[int, int, int], float]:
    """Timing function for one batched launch over the frames of `table`."""
    return _measure_with(det, lambda: det.detect_batched(None, table=table, **kw), reps)


def tune_detector_frame(det, frame, n_sm: Optional[int] = None, cache_path: Optional[str] = None) -> TuneResult:
    """Pick and apply the band height for single frames shaped like `frame`."""
    import torch
    n_sm = n_sm or torch.cuda.get_device_properties(frame.device).multi_processor_count
    t = Autotuner(n_sm, det.radii, cache_path)
    res = t.tune([tuple(frame.shape[-2:])], frame_measure(det, frame), mode="frame")
    det.set_producer_warps(res.producer_warps)
    det.set_tiling(res.band, res.ctas_per_sm)
    return res


def tune_detector_batch(det, table, shapes, n_sm: Optional[int] = None, cache_path: Optional[str] = None,
                        **kw) -> TuneResult:
    """Pick and apply the band height for batched launches over `shapes`."""
    import torch
    n_sm = n_sm or torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    t = Autotuner(n_sm, det.radii, cache_path)
    res = t.tune(list(shapes), batch_measure(det, table, **kw), mode="batch")
    det.set_producer_warps(res.producer_warps)
    det.set_tiling(res.band, res.ctas_per_sm)
    return res
