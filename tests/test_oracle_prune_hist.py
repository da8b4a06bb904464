"""Pins of the oracle's overlap pruning (Sec. 4.1), disc overlap, volume
histogram (Sec. 4) and the differentiable soft histogram."""
import math

import numpy as np
import pytest

import oracle
from paper_2010_08486_gb300 import synth

CFG1 = oracle.OracleParams(min_sigma=1.0, max_sigma=10.0, ratio=1.6, threshold=0.1)


# ------------------------------------------------------------------- overlap

def _grid_overlap(x1, y1, r1, x2, y2, r2, n=2000):
    # midpoint-rule area of the intersection on a fine grid over the smaller disc
    rmin = min(r1, r2)
    cx, cy = (x1, y1) if r1 <= r2 else (x2, y2)
    ox, oy, orr = (x2, y2, r2) if r1 <= r2 else (x1, y1, r1)
    t = (np.arange(n) + 0.5) / n * 2 * rmin - rmin
    X, Y = np.meshgrid(t + cx, t + cy)
    inside_small = (X - cx) ** 2 + (Y - cy) ** 2 <= rmin ** 2
    inside_other = (X - ox) ** 2 + (Y - oy) ** 2 <= orr ** 2
    cell = (2 * rmin / n) ** 2
    return np.sum(inside_small & inside_other) * cell / (math.pi * rmin ** 2)


@pytest.mark.parametrize("case", [(0, 0, 3.0, 2, 1, 3.0), (0, 0, 5.0, 4, 3, 2.0),
                                  (0, 0, 1.5, 2, 0, 2.5), (0, 0, 8.0, 7, 7, 6.0)])
def test_overlap_matches_area_integration(case):
    got = oracle.overlap(*case)
    want = _grid_overlap(*case)
    assert abs(got - want) < 1e-3


def test_overlap_equal_radii_closed_form():
    # equal discs: lens area 2 r^2 acos(d / 2r) - (d / 2) sqrt(4 r^2 - d^2)
    for r in (1.0, 2.5, 7.0):
        for d in np.linspace(0.1, 2 * r - 0.1, 7):
            lens = 2 * r * r * math.acos(d / (2 * r)) - 0.5 * d * math.sqrt(4 * r * r - d * d)
            assert abs(oracle.overlap(0, 0, r, d, 0, r) - lens / (math.pi * r * r)) < 1e-12


def test_overlap_limits_and_symmetry():
    assert oracle.overlap(3, 4, 2.0, 3, 4, 2.0) == 1.0
    assert oracle.overlap(0, 0, 5.0, 1, 1, 2.0) == 1.0          # containment
    assert oracle.overlap(0, 0, 1.0, 3, 0, 2.0) == 0.0          # touching
    assert oracle.overlap(0, 0, 1.0, 10, 0, 2.0) == 0.0
    a = oracle.overlap(0, 0, 3.0, 2, 2, 4.0)
    b = oracle.overlap(2, 2, 4.0, 0, 0, 3.0)
    assert a == b and 0 < a < 1


# --------------------------------------------------------------------- prune

def _blobs(rows):
    a = np.array(rows, dtype=np.float64).reshape(-1, 4)
    return oracle.Blobs(a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int32),
                        np.zeros(len(a)), a[:, 3])


def test_prune_hand_cases():
    sig = oracle.ladder(CFG1)            # 1, 1.6, 2.56, 4.096, 6.55, 10.49
    p = CFG1
    # two same-level blobs 2 px apart at sigma 4.096 (r = 5.79): merged,
    # the stronger one's centre survives with its own ladder sigma
    out = oracle.prune(_blobs([(10, 10, 3, 0.5), (12, 10, 3, 0.9)]), p)
    assert len(out) == 1 and (out.x[0], out.y[0]) == (12, 10) and out.sigma[0] == sig[3]
    # far apart: both kept, in response order
    out = oracle.prune(_blobs([(10, 10, 3, 0.5), (80, 10, 3, 0.9)]), p)
    assert list(out.x) == [80, 10]
    # chain A > B > C with B overlapping A and C overlapping B but not A:
    # B joins A, C is compared with accepted blobs only and survives
    out = oracle.prune(_blobs([(0, 0, 2, 0.9), (2, 0, 2, 0.8), (4, 0, 2, 0.7)]), p)
    assert oracle.overlap(0, 0, math.sqrt(2) * sig[2], 2, 0, math.sqrt(2) * sig[2]) > 0.5
    assert oracle.overlap(2, 0, math.sqrt(2) * sig[2], 4, 0, math.sqrt(2) * sig[2]) > 0.5
    assert oracle.overlap(0, 0, math.sqrt(2) * sig[2], 4, 0, math.sqrt(2) * sig[2]) < 0.5
    assert list(zip(out.x, out.y)) == [(0, 0), (4, 0)]
    # mixed levels coalesce to the mean sigma, summed in visiting order
    out = oracle.prune(_blobs([(20, 20, 3, 0.9), (21, 20, 4, 0.8)]), p)
    assert len(out) == 1 and out.sigma[0] == (sig[3] + sig[4]) / 2
    # equal responses: ties broken by (level, y, x)
    out = oracle.prune(_blobs([(5, 5, 3, 0.5), (4, 5, 3, 0.5)]), p)
    assert (out.x[0], out.y[0]) == (4, 5)


def test_prune_modes():
    rows = [(20, 20, 3, 0.9), (21, 20, 4, 0.8), (90, 90, 1, 0.3)]
    sig = oracle.ladder(CFG1)
    sup = oracle.prune(_blobs(rows), oracle.OracleParams(**{**CFG1.__dict__, "prune": oracle.PRUNE_SUPPRESS}))
    assert list(sup.x) == [20, 90] and sup.sigma[0] == sig[3]
    off = oracle.prune(_blobs(rows), oracle.OracleParams(**{**CFG1.__dict__, "prune": oracle.PRUNE_OFF}))
    assert len(off) == 3 and list(off.response) == [0.9, 0.8, 0.3]


def _lfmis_reference(b, p):
    # Independent formulation: the greedy outcome is the lexicographically
    # first maximal independent set of the conflict graph (overlap > thr) in
    # priority order; every other blob joins its first accepted neighbour.
    sig = oracle.ladder(p)
    n = len(b)
    order = sorted(range(n), key=lambda i: (-b.response[i], b.level[i], b.y[i], b.x[i]))
    rank = {i: k for k, i in enumerate(order)}
    nbr = [[] for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i != j and oracle.overlap(b.x[i], b.y[i], math.sqrt(2) * sig[b.level[i]],
                                         b.x[j], b.y[j], math.sqrt(2) * sig[b.level[j]]) > p.overlap:
                nbr[i].append(j)
    state = {}
    while len(state) < n:
        for i in order:
            if i in state:
                continue
            higher = [j for j in nbr[i] if rank[j] < rank[i]]
            if any(state.get(j) == "in" for j in higher):
                state[i] = "out"
            elif all(state.get(j) == "out" for j in higher):
                state[i] = "in"
    groups = {i: [i] for i in order if state[i] == "in"}
    for i in order:
        if state[i] == "out":
            target = min((j for j in nbr[i] if state[j] == "in"), key=lambda j: rank[j])
            groups[target].append(i)
    res = {}
    for a, members in groups.items():
        levels = {int(b.level[m]) for m in members}
        if len(levels) == 1:
            s = sig[b.level[a]]
        else:
            s = 0.0
            for m in sorted(members, key=lambda m: rank[m]):
                s += sig[b.level[m]]
            s /= len(members)
        res[(int(b.level[a]), int(b.y[a]), int(b.x[a]))] = s
    return res


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_prune_equals_independent_lfmis(seed):
    rng = np.random.default_rng(seed)
    n = 60
    rows = [(rng.integers(0, 40), rng.integers(0, 40), rng.integers(0, 5), rng.integers(1, 6) / 5.0)
            for _ in range(n)]
    # drop duplicate positions at the same level
    seen, uniq = set(), []
    for r in rows:
        if (r[0], r[1], r[2]) not in seen:
            seen.add((r[0], r[1], r[2]))
            uniq.append(r)
    b = _blobs(uniq)
    got = oracle.prune(b, CFG1)
    want = _lfmis_reference(b, CFG1)
    assert {(int(l), int(y), int(x)): s for l, y, x, s in zip(got.level, got.y, got.x, got.sigma)} == want


# ----------------------------------------------------------------- histogram

def test_volume_closed_form():
    assert abs(oracle.volume(1.0) - 4.0 / 3.0 * math.pi * 2 ** 1.5) < 1e-12
    assert abs(oracle.volume(3.0) / oracle.volume(1.0) - 27.0) < 1e-12


def test_hist_bins_on_and_off_ladder():
    p = CFG1
    sig = oracle.ladder(p)                 # 6 levels, 5 DoG planes, last plane sigma_4
    # on-ladder bins are floor(32 l / 4) = 8 l (clamped at 31): exact edges
    assert [oracle.bin_of(np.float32(sig[l]), l, p) for l in range(5)] == [0, 8, 16, 24, 31]
    # off-ladder: t = 0.3 of the log-volume range gives bin floor(9.6) = 9
    s = sig[0] * 1.6 ** (0.3 * 4)
    assert oracle.bin_of(np.float32(s), 1, p) == 9
    # LADDER mode: on-ladder -> own plane; off-ladder -> nearest plane in log sigma
    pl = oracle.OracleParams(**{**p.__dict__, "hist_mode": oracle.HIST_LADDER})
    assert [oracle.bin_of(np.float32(sig[l]), l, pl) for l in range(5)] == [0, 1, 2, 3, 4]
    assert oracle.bin_of(np.float32(sig[2] * 1.6 ** 0.4), 1, pl) == 2
    assert oracle.bin_of(np.float32(sig[2] * 1.6 ** 0.6), 1, pl) == 3


def test_hist_sums_and_volumes():
    img = synth.small_blob_frame(1).astype(np.float64)
    det = oracle.detect(img, CFG1)
    assert int(det.counts.sum()) == len(det.blobs)
    want_vol = sum(4 / 3 * math.pi * (math.sqrt(2) * float(np.float32(s))) ** 3 for s in det.blobs.sigma)
    assert abs(det.volumes.sum() - want_vol) < 1e-9 * want_vol


# ------------------------------------------------------------ soft histogram

CFG4 = oracle.OracleParams(min_sigma=1.0, ratio=1.25, n_levels=12, threshold=0.05, soft_T=0.01)


def _crop():
    frame = synth.plif_frame(synth.GRAD_SEED_BASE)
    return frame[480:544, 480:544].astype(np.float64)


def test_soft_hist_partition_of_unity():
    # the triangular weights of one plane sum to 1, so the histogram mass is
    # the sum of sigmoid((D - thr)/T) over the hard local maxima
    img = _crop()
    sig = oracle.ladder(CFG4)
    rad = oracle.radii(sig, 4.0)
    H = oracle.soft_hist(img, sig, rad, CFG4, sig)
    D = oracle.dog(img, sig, rad)
    import scipy.ndimage as ndi
    mx = ndi.maximum_filter(D, size=3, mode="constant", cval=-np.inf)
    m = D == mx
    want = np.sum(1.0 / (1.0 + np.exp(-(D[m] - 0.05) / 0.01)))
    assert abs(H.sum() - want) < 1e-9 * want


def test_soft_hist_single_blob_lands_in_its_bins():
    p = oracle.OracleParams(min_sigma=1.0, ratio=1.25, n_levels=12, threshold=0.05, soft_T=0.01)
    sig = oracle.ladder(p)
    rad = oracle.radii(sig, 4.0)
    j = 6
    s = sig[j] * math.sqrt(1.25)
    img = synth.isolated_blob_frame(129, 129, [(64, 64)], s, 1.0)
    H = oracle.soft_hist(img, sig, rad, p, sig)
    t = (math.log(sig[j]) - math.log(sig[0])) / (math.log(sig[10]) - math.log(sig[0]))
    b = int(math.floor(32 * t - 0.5))
    assert H[b] + H[b + 1] > 0.9
    assert abs(H[b] / (H[b] + H[b + 1]) - (1 - (32 * t - 0.5 - b))) < 0.05


def test_soft_grad_matches_central_differences():
    # FP64 central differences (h = 1e-6) with the mask frozen, on the 64x64
    # crop at (480, 480) of the first differentiable-workload frame.
    img = _crop()
    sig0 = oracle.ladder(CFG4)
    rad = oracle.radii(sig0, 4.0)
    p = CFG4
    target_img = synth.plif_frame(synth.GRAD_TARGET_SEED_BASE)[480:544, 480:544].astype(np.float64)
    target = oracle.soft_hist(target_img, sig0, rad, p, sig0)
    sig = sig0 * (1.0 + 0.01 * np.sin(np.arange(len(sig0))))
    D = oracle.dog(img, sig, rad)
    mask = oracle.max_mask(D)
    H = oracle.soft_hist(img, sig, rad, p, sig0, mask)
    gH = 2.0 * (H - target)
    gi, gs = oracle.soft_grad(img, sig, rad, p, sig0, gH, mask)
    h = 1e-6

    def loss(im, sg):
        return oracle.soft_loss(im, sg, rad, p, sig0, target, mask)

    fd_s = np.zeros(len(sig))
    for k in range(len(sig)):
        e = np.zeros(len(sig))
        e[k] = h
        fd_s[k] = (loss(img, sig + e) - loss(img, sig - e)) / (2 * h)
    assert np.linalg.norm(fd_s - gs) <= 1e-6 * np.linalg.norm(gs)
    rng = np.random.default_rng(0)
    # pixels with the largest gradient plus random ones
    flat = np.argsort(-np.abs(gi).ravel())[:24].tolist() + rng.integers(0, gi.size, 16).tolist()
    fd_i, an_i = [], []
    for q in flat:
        y, x = divmod(q, gi.shape[1])
        e = np.zeros_like(img)
        e[y, x] = h
        fd_i.append((loss(img + e, sig) - loss(img - e, sig)) / (2 * h))
        an_i.append(gi[y, x])
    fd_i, an_i = np.array(fd_i), np.array(an_i)
    assert np.linalg.norm(fd_i - an_i) <= 1e-6 * np.linalg.norm(an_i)
