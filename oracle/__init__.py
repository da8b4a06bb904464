"""FP64 CPU oracle for DoG blob detection (arXiv 2010.08486, Sec. 3-4).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It is independent of the CUDA path: it shares no code, header, table
or helper with ``paper_2010_08486_gb300`` and never imports it.

The arithmetic lives in ``dog_oracle.c`` (plain double-precision loops); this
module compiles it with gcc on first use and wraps it with ctypes.  Functions
cite the passage they restate.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, scipy, brute force or invariants; see the design notes
for the list.  Nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dog_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

LADDER_GEOM, LADDER_ARITH = 0, 1
NORM_DERIV, NORM_PAPER = 0, 1
PRUNE_COALESCE, PRUNE_SUPPRESS, PRUNE_OFF = 0, 1, 2
HIST_LOGV, HIST_LADDER = 0, 1


def build(force: bool = False) -> str:
    """Compile dog_oracle.c into _build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    # -ffp-contract=off: every a*b+c rounds twice, as written, on every host
    # (gcc for aarch64 would otherwise fuse them), so the oracle gives the same
    # doubles on x86-64 and Arm; no -march=native for the same reason.
    cmd = ["gcc", "-O3", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i, u8 = ctypes.c_double, ctypes.c_int, ctypes.c_uint8
        dp, ip, i32p = P(d), P(i), P(ctypes.c_int32)
        u16p = P(ctypes.c_uint16)
        lib.ora_stretch_rank.argtypes = [ctypes.c_long, d]
        lib.ora_stretch_rank.restype = ctypes.c_long
        lib.ora_stretch_limits.argtypes = [u16p, ctypes.c_long, d, i32p, i32p]
        lib.ora_stretch_limits.restype = i
        lib.ora_stretch.argtypes = [u16p, ctypes.c_long, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_float)]
        u32p = P(ctypes.c_uint32)
        lib.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.ora_render_spheres.argtypes = [P(ctypes.c_float), i, i, i, i, ctypes.c_float, d, d, ctypes.c_uint64,
                                           P(ctypes.c_float), u16p]
        lib.ora_render_spheres.restype = i
        lib.ora_num_threads.restype = i
        lib.ora_reflect.argtypes = [ctypes.c_long, ctypes.c_long]
        lib.ora_reflect.restype = ctypes.c_long
        lib.ora_ladder_geom_count.argtypes = [d, d, d]
        lib.ora_ladder_geom_count.restype = i
        lib.ora_ladder_geom.argtypes = [d, d, i, dp]
        lib.ora_ladder_arith.argtypes = [d, d, i, dp]
        lib.ora_radius.argtypes = [d, d]
        lib.ora_radius.restype = i
        lib.ora_gauss_kernel.argtypes = [d, i, dp]
        lib.ora_gauss_kernel_dsigma.argtypes = [d, i, dp]
        lib.ora_blur2.argtypes = [dp, i, i, dp, dp, i, dp]
        lib.ora_blur.argtypes = [dp, i, i, d, i, dp]
        lib.ora_blur2_adjoint.argtypes = [dp, i, i, dp, dp, i, dp]
        lib.ora_norm_coeffs.argtypes = [dp, i, i, dp]
        lib.ora_dog.argtypes = [dp, i, i, dp, ip, i, i, dp]
        lib.ora_local_max.argtypes = [dp, i, i, i, d, i, i32p, dp, i]
        lib.ora_local_max.restype = i
        lib.ora_overlap.argtypes = [d, d, d, d, d, d]
        lib.ora_overlap.restype = d
        lib.ora_prune.argtypes = [i, i32p, i32p, i32p, dp, dp, d, i, i32p, i32p, i32p, dp, dp]
        lib.ora_prune.restype = i
        lib.ora_volume.argtypes = [d]
        lib.ora_volume.restype = d
        lib.ora_bin.argtypes = [ctypes.c_float, i, dp, i, i, i, i]
        lib.ora_bin.restype = i
        lib.ora_hist.argtypes = [i, P(ctypes.c_float), i32p, dp, i, i, i, i, P(ctypes.c_uint32), dp]
        lib.ora_max_mask.argtypes = [dp, i, i, i, P(u8)]
        lib.ora_soft_hist.argtypes = [dp, i, i, dp, ip, i, i, d, d, i, d, d, P(u8), dp]
        lib.ora_soft_grad.argtypes = [dp, i, i, dp, ip, i, i, d, d, i, d, d, P(u8), dp, dp, dp]
        _lib = lib
        return lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(_load().ora_num_threads())


# ---------------------------------------------------------------- parameters

@dataclasses.dataclass
class OracleParams:
    """Detector hyper-parameters (Sec. 4: n_bin, min_sigma, max_sigma;
    Sec. 4.1: truncate, threshold 0.1, overlap 0.5)."""
    min_sigma: float = 1.0
    max_sigma: float = 10.0
    ratio: float = 1.6
    n_levels: int = 0            # 0: derive from max_sigma
    ladder: int = LADDER_GEOM
    sigmas: tuple | None = None  # explicit ladder overrides the above
    truncate: float = 4.0
    threshold: float = 0.1
    overlap: float = 0.5
    norm: int = NORM_DERIV
    prune: int = PRUNE_COALESCE
    nbins: int = 32
    hist_mode: int = HIST_LOGV
    soft_T: float = 0.01

    def ladder_sigmas(self) -> np.ndarray:
        return ladder(self)

    def is_geom(self) -> bool:
        return self.sigmas is None and self.ladder == LADDER_GEOM


def ladder(p: OracleParams) -> np.ndarray:
    """sigma ladder: explicit, geometric, or Eq. 1 (arithmetic)."""
    lib = _load()
    if p.sigmas is not None:
        return _f64(p.sigmas).copy()
    if p.ladder == LADDER_ARITH:
        K = int(p.n_levels)
        out = np.empty(K, np.float64)
        lib.ora_ladder_arith(p.min_sigma, p.max_sigma, K, _p(out, ctypes.c_double))
        return out
    K = int(p.n_levels) if p.n_levels > 0 else int(lib.ora_ladder_geom_count(p.min_sigma, p.max_sigma, p.ratio))
    out = np.empty(K, np.float64)
    lib.ora_ladder_geom(p.min_sigma, p.ratio, K, _p(out, ctypes.c_double))
    return out


def radius(sigma: float, truncate: float) -> int:
    """Sec. 4.1: radius = truncate * sigma, rounded half up."""
    return int(_load().ora_radius(float(sigma), float(truncate)))


def radii(sig, truncate: float) -> np.ndarray:
    return np.array([radius(s, truncate) for s in sig], dtype=np.int32)


def reflect(i: int, n: int) -> int:
    return int(_load().ora_reflect(int(i), int(n)))


def gauss_kernel(sigma: float, r: int) -> np.ndarray:
    """Sampled Gaussian of std sigma on -r..r, normalised to sum 1 (Sec. 3)."""
    out = np.empty(2 * r + 1, np.float64)
    _load().ora_gauss_kernel(float(sigma), int(r), _p(out, ctypes.c_double))
    return out


def gauss_kernel_dsigma(sigma: float, r: int) -> np.ndarray:
    out = np.empty(2 * r + 1, np.float64)
    _load().ora_gauss_kernel_dsigma(float(sigma), int(r), _p(out, ctypes.c_double))
    return out


def blur2(img, kx, ky) -> np.ndarray:
    """Separable reflect-boundary correlation with kx along rows, ky along columns."""
    img = _f64(img)
    kx, ky = _f64(kx), _f64(ky)
    r = (len(kx) - 1) // 2
    assert len(ky) == len(kx)
    h, w = img.shape
    out = np.empty_like(img)
    _load().ora_blur2(_p(img, ctypes.c_double), h, w, _p(kx, ctypes.c_double),
                      _p(ky, ctypes.c_double), r, _p(out, ctypes.c_double))
    return out


def blur(img, sigma: float, r: int) -> np.ndarray:
    """Scale-space level L = g(sigma) * I (Sec. 3)."""
    img = _f64(img)
    h, w = img.shape
    out = np.empty_like(img)
    _load().ora_blur(_p(img, ctypes.c_double), h, w, float(sigma), int(r), _p(out, ctypes.c_double))
    return out


def blur2_adjoint(a, kx, ky) -> np.ndarray:
    a = _f64(a)
    kx, ky = _f64(kx), _f64(ky)
    r = (len(kx) - 1) // 2
    h, w = a.shape
    out = np.zeros_like(a)
    _load().ora_blur2_adjoint(_p(a, ctypes.c_double), h, w, _p(kx, ctypes.c_double),
                              _p(ky, ctypes.c_double), r, _p(out, ctypes.c_double))
    return out


def norm_coeffs(sig, norm: int) -> np.ndarray:
    """Eq. 3 (PAPER) or the heat-equation finite difference (DERIV)."""
    sig = _f64(sig)
    out = np.empty(max(len(sig), 1), np.float64)
    _load().ora_norm_coeffs(_p(sig, ctypes.c_double), len(sig), int(norm), _p(out, ctypes.c_double))
    return out[:len(sig) - 1]


def dog(img, sig, rad, norm: int = NORM_DERIV) -> np.ndarray:
    """Eq. 2-3: D_i = c_i (L_i - L_{i+1}); returns (K-1, h, w) float64."""
    img = _f64(img)
    sig = _f64(sig)
    rad = np.ascontiguousarray(rad, dtype=np.intc)
    h, w = img.shape
    K = len(sig)
    D = np.empty((K - 1, h, w), np.float64)
    _load().ora_dog(_p(img, ctypes.c_double), h, w, _p(sig, ctypes.c_double), _p(rad, ctypes.c_int),
                    K, int(norm), _p(D, ctypes.c_double))
    return D


def local_max(D, thr: float, use_thr: bool = True, cap: int | None = None):
    """Sec. 4 / 4.1 maximum-filter test; returns (lyx int32 (n,3), resp float64 (n,))."""
    D = _f64(D)
    P, h, w = D.shape
    if cap is None:
        cap = P * h * w if not use_thr else max(1024, P * h * w // 8)
    lyx = np.empty((cap, 3), np.int32)
    resp = np.empty(cap, np.float64)
    n = _load().ora_local_max(_p(D, ctypes.c_double), P, h, w, float(thr), int(use_thr),
                              _p(lyx, ctypes.c_int32), _p(resp, ctypes.c_double), int(cap))
    if n > cap:
        return local_max(D, thr, use_thr, cap=n)
    return lyx[:n].copy(), resp[:n].copy()


def overlap(x1, y1, r1, x2, y2, r2) -> float:
    return float(_load().ora_overlap(float(x1), float(y1), float(r1), float(x2), float(y2), float(r2)))


def volume(sigma: float) -> float:
    """r = sqrt(2) sigma, V = 4/3 pi r^3 (Sec. 4)."""
    return float(_load().ora_volume(float(sigma)))


@dataclasses.dataclass
class Blobs:
    """Blob list (x = column, y = row, DoG plane index, sigma, response)."""
    x: np.ndarray
    y: np.ndarray
    level: np.ndarray
    sigma: np.ndarray
    response: np.ndarray

    def __len__(self) -> int:
        return int(len(self.x))

    def canonical(self) -> "Blobs":
        """Sorted by (level, y, x)."""
        order = np.lexsort((self.x, self.y, self.level))
        return Blobs(self.x[order], self.y[order], self.level[order], self.sigma[order],
                     self.response[order])

    def keys(self) -> set:
        return set(zip(self.level.tolist(), self.y.tolist(), self.x.tolist()))


def candidates(img, p: OracleParams, D: np.ndarray | None = None) -> Blobs:
    """Thresholded 3x3x3 local maxima of the DoG cube, sigma = ladder sigma."""
    sig = ladder(p)
    if D is None:
        D = dog(img, sig, radii(sig, p.truncate), p.norm)
    lyx, resp = local_max(D, p.threshold, True)
    lev = lyx[:, 0].astype(np.int32)
    return Blobs(lyx[:, 2].astype(np.int32), lyx[:, 1].astype(np.int32), lev,
                 sig[lev] if len(lev) else np.zeros(0), resp)


def prune(c: Blobs, p: OracleParams) -> Blobs:
    """Sec. 4.1 overlap pruning (see dog_oracle.c ora_prune)."""
    sig = ladder(p)
    n = len(c)
    x, y, lev = _i32(c.x), _i32(c.y), _i32(c.level)
    resp = _f64(c.response)
    ox, oy, ol = (np.empty(max(n, 1), np.int32) for _ in range(3))
    os_, orr = np.empty(max(n, 1), np.float64), np.empty(max(n, 1), np.float64)
    m = _load().ora_prune(n, _p(x, ctypes.c_int32), _p(y, ctypes.c_int32), _p(lev, ctypes.c_int32),
                          _p(resp, ctypes.c_double), _p(sig, ctypes.c_double), float(p.overlap),
                          int(p.prune), _p(ox, ctypes.c_int32), _p(oy, ctypes.c_int32),
                          _p(ol, ctypes.c_int32), _p(os_, ctypes.c_double), _p(orr, ctypes.c_double))
    return Blobs(ox[:m].copy(), oy[:m].copy(), ol[:m].copy(), os_[:m].copy(), orr[:m].copy())


def bin_of(sigma_f32: float, level: int, p: OracleParams) -> int:
    sig = ladder(p)
    return int(_load().ora_bin(ctypes.c_float(np.float32(sigma_f32)), int(level), _p(sig, ctypes.c_double),
                               len(sig), int(p.is_geom()), int(p.nbins), int(p.hist_mode)))


def hist(b: Blobs, p: OracleParams):
    """Counts and summed volume per bin; sigma is taken as stored (single)."""
    sig = ladder(p)
    n = len(b)
    sf = np.ascontiguousarray(b.sigma, dtype=np.float32)
    lev = _i32(b.level)
    nb = (len(sig) - 1) if p.hist_mode == HIST_LADDER else p.nbins
    counts = np.zeros(nb, np.uint32)
    vol = np.zeros(nb, np.float64)
    _load().ora_hist(n, _p(sf, ctypes.c_float), _p(lev, ctypes.c_int32), _p(sig, ctypes.c_double),
                     len(sig), int(p.is_geom()), int(p.nbins), int(p.hist_mode),
                     _p(counts, ctypes.c_uint32), _p(vol, ctypes.c_double))
    return counts, vol


@dataclasses.dataclass
class Detection:
    candidates: Blobs
    blobs: Blobs
    counts: np.ndarray
    volumes: np.ndarray
    D: np.ndarray | None = None


def detect(img, p: OracleParams, keep_dog: bool = False) -> Detection:
    """Whole method of Sec. 4: scale space, DoG, 3x3x3 maxima above the
    threshold, overlap pruning, volume histogram."""
    sig = ladder(p)
    D = dog(img, sig, radii(sig, p.truncate), p.norm)
    c = candidates(img, p, D=D)
    b = prune(c, p)
    b.sigma = b.sigma.astype(np.float32).astype(np.float64)
    counts, vol = hist(b, p)
    return Detection(c, b, counts, vol, D if keep_dog else None)


# ------------------------------------------------ differentiable soft histogram

def max_mask(D) -> np.ndarray:
    D = _f64(D)
    P, h, w = D.shape
    m = np.empty((P, h, w), np.uint8)
    _load().ora_max_mask(_p(D, ctypes.c_double), P, h, w, _p(m, ctypes.c_uint8))
    return m


def soft_hist(img, sig, rad, p: OracleParams, sref, mask=None) -> np.ndarray:
    """Soft blob-volume histogram over the hard local maxima (no threshold)."""
    img = _f64(img)
    sig = _f64(sig)
    rad = np.ascontiguousarray(rad, dtype=np.intc)
    sref = _f64(sref)
    h, w = img.shape
    H = np.zeros(p.nbins, np.float64)
    mp = None if mask is None else _p(np.ascontiguousarray(mask, dtype=np.uint8), ctypes.c_uint8)
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        mp = _p(mask, ctypes.c_uint8)
    _load().ora_soft_hist(_p(img, ctypes.c_double), h, w, _p(sig, ctypes.c_double),
                          _p(rad, ctypes.c_int), len(sig), int(p.norm), float(p.threshold),
                          float(p.soft_T), int(p.nbins), float(sref[0]), float(sref[len(sref) - 2]),
                          mp, _p(H, ctypes.c_double))
    return H


def soft_grad(img, sig, rad, p: OracleParams, sref, gH, mask=None):
    """(grad_img, grad_sigma) of a loss with dloss/dH = gH through soft_hist."""
    img = _f64(img)
    sig = _f64(sig)
    rad = np.ascontiguousarray(rad, dtype=np.intc)
    sref = _f64(sref)
    gH = _f64(gH)
    h, w = img.shape
    gi = np.zeros((h, w), np.float64)
    gs = np.zeros(len(sig), np.float64)
    mp = None
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        mp = _p(mask, ctypes.c_uint8)
    _load().ora_soft_grad(_p(img, ctypes.c_double), h, w, _p(sig, ctypes.c_double),
                          _p(rad, ctypes.c_int), len(sig), int(p.norm), float(p.threshold),
                          float(p.soft_T), int(p.nbins), float(sref[0]), float(sref[len(sref) - 2]),
                          mp, _p(gH, ctypes.c_double), _p(gi, ctypes.c_double), _p(gs, ctypes.c_double))
    return gi, gs


def soft_loss(img, sig, rad, p: OracleParams, sref, target, mask=None) -> float:
    """Squared error of the soft histogram against a target histogram."""
    H = soft_hist(img, sig, rad, p, sref, mask)
    return float(np.sum((H - np.asarray(target, np.float64)) ** 2))


def continuum_peak_response(amp: float, ratio: float) -> float:
    """Closed form: with c_i = 1/(r-1) on a geometric ladder, the response at the
    centre of a Gaussian blob of std s is A s^2 sig^2 (r+1) / ((s^2+sig^2)(s^2+r^2 sig^2)),
    maximal at sig = s / sqrt(r) with value A / (r + 1)."""
    return amp / (ratio + 1.0)


def continuum_centre_response(amp: float, s: float, sig: float, ratio: float) -> float:
    return amp * s * s * sig * sig * (ratio + 1.0) / ((s * s + sig * sig) * (s * s + ratio * ratio * sig * sig))



# ---------------------------------------------------------------------------
# Preprocessing: contrast stretch with saturation (Sec. 4, first, optional
# step; 0.35% in the paper).

def stretch_rank(n: int, sat: float) -> int:
    """k = floor(sat / 2 * n): the rank (0-based, ascending) of the count that
    maps to 0; rank n - 1 - k maps to 1."""
    return int(_load().ora_stretch_rank(int(n), float(sat)))


def stretch_limits(counts, sat: float = 0.0035):
    """(lo, hi) of a frame of 12-bit counts (values above 4095 count as 4095):
    the counts at ranks k and n - 1 - k of the sorted frame."""
    c = np.ascontiguousarray(counts, dtype=np.uint16).ravel()
    lo, hi = ctypes.c_int32(), ctypes.c_int32()
    rc = _load().ora_stretch_limits(c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), c.size, float(sat),
                                   ctypes.byref(lo), ctypes.byref(hi))
    if rc != 0:
        raise ValueError("stretch_limits failed (%d)" % rc)
    return lo.value, hi.value


def stretch(counts, lo: int, hi: int) -> np.ndarray:
    """The stretched frame in [0, 1] (float32): (c - lo) / (hi - lo) in double,
    clipped, rounded to float."""
    c = np.ascontiguousarray(counts, dtype=np.uint16)
    out = np.empty(c.shape, dtype=np.float32)
    _load().ora_stretch(c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), c.size, int(lo), int(hi),
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


def preprocess(counts, sat: float = 0.0035) -> np.ndarray:
    """Contrast-stretched frame with the frame's own limits."""
    lo, hi = stretch_limits(counts, sat)
    return stretch(counts, lo, hi)


# ---------------------------------------------------------------------------
# Synthetic sphere frames (Sec. 5: 100 rendered spheres with Poisson and
# Gaussian noise); the shading reading is stated in dog_oracle.c.

def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) of a 4-word counter and a
    2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    _load().ora_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def render_spheres(spheres, h: int, w: int, ss: int = 4, background: float = 0.05, gain: float = 2000.0,
                   read_noise: float = 4.0, seed: int = 0):
    """(intensity (h, w) float32, counts (h, w) uint16) of a sphere table
    (S, 4): cx, cy, R, A."""
    sp = np.ascontiguousarray(spheres, dtype=np.float32).reshape(-1, 4)
    inten = np.empty((h, w), dtype=np.float32)
    counts = np.empty((h, w), dtype=np.uint16)
    rc = _load().ora_render_spheres(sp.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), sp.shape[0], h, w, ss,
                                    float(background), float(gain), float(read_noise), int(seed),
                                    inten.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    if rc != 0:
        raise ValueError("render_spheres failed (%d)" % rc)
    return inten, counts
