"""Tile-shape autotuner: model, candidate ranking, selection and cache, on
the CPU with an injected timing function."""
import math

import pytest

from paper_2010_08486_gb300 import autotune

# radii of the 25-level ladder sigma = 0.8 * 1.1^i, truncate 4
RADII = [int(math.floor(4.0 * 0.8 * 1.1 ** i + 0.5)) for i in range(25)]


def test_warmup_rows_of_plif_ladder():
    assert RADII[0] == 3 and RADII[-1] == 32
    assert autotune.warmup_rows(RADII) == 72     # 8 * ceil(65 / 8)


def test_tiles_and_model_cost():
    assert autotune.tiles_of((1024, 1024), 0) == 32
    assert autotune.tiles_of((1024, 1024), 256) == 128
    assert autotune.tiles_of((1000, 33), 256) == 8
    # whole frames: one wave of 32 strips of 1024 rows + 2 + half the warm-up
    assert autotune.model_cost([(1024, 1024)], 0, RADII, 152) == pytest.approx(1024 + 2 + 36)
    # 4 bands: 128 tiles, still one wave
    assert autotune.model_cost([(1024, 1024)], 256, RADII, 152) == pytest.approx(256 + 2 + 36)
    # 8 bands: 256 tiles, two waves
    assert autotune.model_cost([(1024, 1024)], 128, RADII, 152) == pytest.approx(2 * (128 + 2 + 36))


def test_candidates_rank_single_frame():
    c = autotune.candidate_bands([(1024, 1024)], RADII, 152, limit=4)
    # the best modelled height: 232 rows (4 full bands + a 96-row band whose
    # 32 short tiles, and the 8 that spill into a second round, finish within
    # the full bands' time) beats 256
    assert c[0] == 232
    best = autotune.model_cost([(1024, 1024)], c[0], RADII, 152)
    assert all(best <= autotune.model_cost([(1024, 1024)], b, RADII, 152) for b in range(8, 1024, 8))
    assert 0 in c
    assert all(b % 8 == 0 for b in c)


def test_tuner_picks_fastest_and_caches(tmp_path):
    calls = []

    def measure(band, cps, nw):
        calls.append((band, cps, nw))
        base = {256: 1.0, 0: 3.0}.get(band, 2.0) if band != 232 else float("inf")
        return base * (0.9 if nw == 8 else 1.0)

    path = str(tmp_path / "tune.json")
    t = autotune.Autotuner(152, RADII, path)
    r = t.tune([(1024, 1024)], measure)
    assert (r.band, r.ctas_per_sm, r.ms, r.producer_warps) == (256, 1, 0.9, 8)
    assert {c[2] for c in calls} == {8, 12}     # both kernel forms timed
    n = len(calls)
    assert t.tune([(1024, 1024)], measure).band == 256
    assert len(calls) == n                 # cached
    t2 = autotune.Autotuner(152, RADII, path)   # reloaded from disk
    r2 = t2.tune([(1024, 1024)], measure)
    assert (r2.band, r2.ms, r2.producer_warps) == (256, 0.9, 8) and len(calls) == n
    # another shape mix is another key
    t.tune([(128, 128), (512, 512)], measure, mode="batch")
    assert len(calls) > n


def test_tuner_all_failed():
    t = autotune.Autotuner(152, RADII)
    with pytest.raises(RuntimeError):
        t.tune([(64, 64)], lambda b, c, w: float("nan"))
