"""Python API of the GB300 DoG blob detector.

Every computation runs in libdog.so's CUDA kernels; this module only
allocates device tensors with PyTorch, passes pointers and sizes through the
C ABI (include/dog.h), and wraps results.  Method: arXiv 2010.08486, Sec. 3-4.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Sequence

import torch

from . import _lib
from ._lib import check


@dataclasses.dataclass
class DetectorConfig:
    """Hyper-parameters of Sec. 4 / 4.1 (see dog_config in include/dog.h)."""
    min_sigma: float = 1.0
    max_sigma: float = 10.0
    ratio: float = 1.6
    n_levels: int = 0
    ladder: int = _lib.LADDER_GEOM
    sigmas: Sequence[float] | None = None
    truncate: float = 4.0
    threshold: float = 0.1
    overlap: float = 0.5
    norm: int = _lib.NORM_DERIV
    prune: int = _lib.PRUNE_COALESCE
    nbins: int = 32
    hist_mode: int = _lib.HIST_LOGV
    soft_T: float = 0.01
    max_h: int = 1024
    max_w: int = 1024
    blob_cap: int = 65536
    stretch_sat: float = 0.0
    backend: int = _lib.BACKEND_DIRECT

    def to_c(self):
        c = _lib.DogConfig()
        _lib.load().dog_config_default(ctypes.byref(c))
        keep = None
        for f in dataclasses.fields(self):
            if f.name == "sigmas":
                continue
            setattr(c, f.name, getattr(self, f.name))
        if self.sigmas is not None:
            keep = (ctypes.c_double * len(self.sigmas))(*[float(s) for s in self.sigmas])
            c.sigmas = ctypes.cast(keep, ctypes.POINTER(ctypes.c_double))
            c.n_levels = len(self.sigmas)
        return c, keep


def small_frame_config(**kw) -> DetectorConfig:
    """256x256 workload: ladder 1.6^i from 1 to 10, threshold 0.1."""
    return DetectorConfig(**{**dict(min_sigma=1.0, max_sigma=10.0, ratio=1.6, threshold=0.1,
                                    max_h=256, max_w=256, blob_cap=65536), **kw})


def plif_config(**kw) -> DetectorConfig:
    """PLIF-shaped 1024x1024 workload: 25 levels 0.8 * 1.1^i, threshold 0.05."""
    return DetectorConfig(**{**dict(min_sigma=0.8, ratio=1.1, n_levels=25, threshold=0.05,
                                    max_h=1024, max_w=1024, blob_cap=65536), **kw})


def grad_config(**kw) -> DetectorConfig:
    """Differentiable workload: 12 sigmas 1.25^k, threshold 0.05, T = 0.01."""
    return DetectorConfig(**{**dict(min_sigma=1.0, ratio=1.25, n_levels=12, threshold=0.05,
                                    soft_T=0.01, max_h=1024, max_w=1024, blob_cap=65536), **kw})


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _img_dtype(img: torch.Tensor) -> int:
    if img.dtype == torch.float32:
        return _lib.DTYPE_F32
    if img.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return _lib.DTYPE_U16
    raise TypeError("frames must be float32 or 16-bit counts, got %s" % img.dtype)


def _check_img(img: torch.Tensor):
    if not img.is_cuda:
        raise ValueError("frame must be a CUDA tensor")
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("frame must be 2-D with unit column stride")
    return img.shape[0], img.shape[1], img.stride(0)


@dataclasses.dataclass
class BlobList:
    """Device blob records: x, y, level (int32), sigma, response (float32)."""
    raw: torch.Tensor      # (cap, 5) int32
    count: torch.Tensor    # () int32 on the device

    def n(self) -> int:
        return int(self.count.item())

    def to_numpy(self):
        n = min(self.n(), self.raw.shape[0])
        r = self.raw[:n].cpu()
        ints = r[:, :3].numpy()
        flt = r[:, 3:].view(torch.float32).numpy()
        return ints[:, 0], ints[:, 1], ints[:, 2], flt[:, 0], flt[:, 1]


def empty_blobs(cap: int, device) -> BlobList:
    return BlobList(torch.empty((cap, 5), dtype=torch.int32, device=device),
                    torch.zeros((), dtype=torch.int32, device=device))


def stretch_limits(counts: torch.Tensor, sat: float = 0.0035, stream=None) -> torch.Tensor:
    """Contrast-stretch limits (lo, hi) of one frame of 12-bit counts (Sec. 4
    preprocessing; dog_stretch_limits): a (2,) int32 device tensor."""
    if _img_dtype(counts) != _lib.DTYPE_U16:
        raise TypeError("the contrast stretch takes 16-bit counts")
    H, W, pitch = _check_img(counts)
    hist = torch.empty(4096, dtype=torch.int32, device=counts.device)
    lohi = torch.empty(2, dtype=torch.int32, device=counts.device)
    check(_lib.load().dog_stretch_limits(counts.data_ptr(), H, W, pitch, float(sat), hist.data_ptr(),
                                         lohi.data_ptr(), _stream(stream)), "dog_stretch_limits")
    return lohi


def stretch(counts: torch.Tensor, lohi: torch.Tensor | None = None, sat: float = 0.0035,
            stream=None) -> torch.Tensor:
    """The stretched FP32 frame in [0, 1] (dog_stretch), with the frame's own
    limits unless `lohi` is given."""
    if lohi is None:
        lohi = stretch_limits(counts, sat, stream)
    H, W, pitch = _check_img(counts)
    out = torch.empty((H, W), dtype=torch.float32, device=counts.device)
    check(_lib.load().dog_stretch(counts.data_ptr(), H, W, pitch, lohi.data_ptr(), out.data_ptr(), W,
                                  _stream(stream)), "dog_stretch")
    return out


def render_spheres(spheres: torch.Tensor, h: int, w: int, ss: int = 4, background: float = 0.05,
                   gain: float = 2000.0, read_noise: float = 4.0, seed: int = 0, with_intensity: bool = False,
                   stream=None):
    """Synthetic frame of rendered spheres (dog_render_spheres): 12-bit counts
    (h, w) as int16 bits (and the noiseless FP32 intensity)."""
    sp = spheres.contiguous()
    if sp.dtype != torch.float32 or sp.dim() != 2 or sp.shape[1] != 4 or not sp.is_cuda:
        raise ValueError("spheres: (n, 4) float32 CUDA tensor (cx, cy, R, A)")
    counts = torch.empty((h, w), dtype=torch.int16, device=sp.device)
    inten = torch.empty((h, w), dtype=torch.float32, device=sp.device) if with_intensity else None
    check(_lib.load().dog_render_spheres(sp.data_ptr() if sp.shape[0] else None, sp.shape[0], h, w, ss,
                                         float(background), float(gain), float(read_noise), int(seed),
                                         _ptr(inten), counts.data_ptr(), w, _stream(stream)),
          "dog_render_spheres")
    return (counts, inten) if with_intensity else counts


class Detector:
    """One handle of the C library on the current CUDA device."""

    def __init__(self, cfg: DetectorConfig | None = None, device=None):
        self.cfg = cfg or DetectorConfig()
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        c, self._keep = self.cfg.to_c()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.dog_create(ctypes.byref(c), ctypes.byref(h)), "dog_create")
        self.h = h
        K = ctypes.c_int32()
        check(self.lib.dog_ladder(self.h, ctypes.byref(K), None, None, None), "dog_ladder")
        self.K = K.value
        self.P = self.K - 1
        sig = (ctypes.c_double * self.K)()
        rad = (ctypes.c_int32 * self.K)()
        nrm = (ctypes.c_double * self.P)()
        check(self.lib.dog_ladder(self.h, None, sig, rad, nrm), "dog_ladder")
        self.sigmas = list(sig)
        self.radii = list(rad)
        self.norm = list(nrm)
        self.nbins_out = self.P if self.cfg.hist_mode == _lib.HIST_LADDER else self.cfg.nbins

    def close(self):
        if getattr(self, "h", None):
            self.lib.dog_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- forward
    def candidates(self, img: torch.Tensor, cap: int | None = None, out: BlobList | None = None,
                   stream=None) -> BlobList:
        H, W, pitch = _check_img(img)
        cap = cap or self.cfg.blob_cap
        out = out or empty_blobs(cap, img.device)
        check(self.lib.dog_candidates(self.h, img.data_ptr(), _img_dtype(img), H, W, pitch,
                                      out.raw.data_ptr(), out.raw.shape[0], out.count.data_ptr(),
                                      _stream(stream)), "dog_candidates")
        return out

    def prune(self, cand: BlobList, H: int, W: int, cap: int | None = None, stream=None) -> BlobList:
        cap = cap or cand.raw.shape[0]
        out = empty_blobs(cap, cand.raw.device)
        check(self.lib.dog_prune(self.h, cand.raw.data_ptr(), cand.count.data_ptr(), cand.raw.shape[0],
                                 H, W, out.raw.data_ptr(), cap, out.count.data_ptr(), _stream(stream)),
              "dog_prune")
        return out

    def volume_hist(self, blobs: BlobList, with_volume: bool = False, stream=None):
        hist = torch.zeros(self.nbins_out, dtype=torch.int32, device=blobs.raw.device)
        vol = torch.zeros(self.nbins_out, dtype=torch.float64, device=blobs.raw.device) if with_volume else None
        check(self.lib.dog_volume_hist(self.h, blobs.raw.data_ptr(), blobs.count.data_ptr(),
                                       blobs.raw.shape[0], hist.data_ptr(), _ptr(vol), _stream(stream)),
              "dog_volume_hist")
        return hist, vol

    def detect(self, img: torch.Tensor, cap: int | None = None, with_volume: bool = False,
               out: BlobList | None = None, hist: torch.Tensor | None = None, stream=None):
        H, W, pitch = _check_img(img)
        cap = cap or self.cfg.blob_cap
        out = out or empty_blobs(cap, img.device)
        if hist is None:
            hist = torch.zeros(self.nbins_out, dtype=torch.int32, device=img.device)
        vol = torch.zeros(self.nbins_out, dtype=torch.float64, device=img.device) if with_volume else None
        check(self.lib.dog_detect(self.h, img.data_ptr(), _img_dtype(img), H, W, pitch,
                                  out.raw.data_ptr(), out.raw.shape[0], out.count.data_ptr(),
                                  hist.data_ptr(), _ptr(vol), _stream(stream)), "dog_detect")
        return out, hist, vol

    def debug_dog(self, img: torch.Tensor, stream=None) -> torch.Tensor:
        H, W, pitch = _check_img(img)
        D = torch.empty((self.P, H, W), dtype=torch.float32, device=img.device)
        check(self.lib.dog_debug_dog(self.h, img.data_ptr(), _img_dtype(img), H, W, pitch, D.data_ptr(),
                                     _stream(stream)), "dog_debug_dog")
        return D

    def set_tiling(self, band_rows: int, ctas_per_sm: int = 1):
        check(self.lib.dog_set_tiling(self.h, band_rows, ctas_per_sm), "dog_set_tiling")

    def set_producer_warps(self, n: int = 0):
        """Kernel form: 8 or 12 producer warps, 0 for the handle's default."""
        check(self.lib.dog_set_producer_warps(self.h, n), "dog_set_producer_warps")

    @property
    def producer_warps(self) -> int:
        return int(self.lib.dog_get_producer_warps(self.h))

    def profile(self, enable: bool = True):
        check(self.lib.dog_profile_enable(self.h, int(enable)), "dog_profile_enable")

    def profile_read(self):
        """(summed fused-kernel milliseconds, launches) since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int32()
        check(self.lib.dog_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n)), "dog_profile_read")
        return ms.value, n.value

    def status(self) -> int:
        v = ctypes.c_int32()
        check(self.lib.dog_get_status(self.h, ctypes.byref(v)), "dog_get_status")
        return v.value

    # ---------------------------------------------------------------- batched
    def frame_table(self, frames: Sequence[torch.Tensor], blob_cap: int | None = None):
        """Device dog_frame table for `frames`; blob slots of blob_cap per frame."""
        cap = blob_cap or self.cfg.blob_cap
        n = len(frames)
        tab = (_lib.DogFrame * n)()
        mh = mw = 0
        for f, img in enumerate(frames):
            H, W, pitch = _check_img(img)
            tab[f].ptr = img.data_ptr()
            tab[f].h, tab[f].w, tab[f].pitch = H, W, pitch
            tab[f].dtype = _img_dtype(img)
            tab[f].blob_off = f * cap
            mh, mw = max(mh, H), max(mw, W)
        host = torch.frombuffer(bytearray(bytes(tab)), dtype=torch.uint8)
        return host.to(frames[0].device), n, mh, mw

    def detect_batched(self, frames: Sequence[torch.Tensor], table=None, out: torch.Tensor | None = None,
                       counts: torch.Tensor | None = None, hists: torch.Tensor | None = None, stream=None):
        """Detect all frames in one persistent launch (+ one prune and one histogram launch).
        Returns (blobs (n*cap, 5) int32, counts (n,), hists (n, nbins))."""
        cap = self.cfg.blob_cap
        tab, n, mh, mw = table if table is not None else self.frame_table(frames, cap)
        dev = tab.device
        out = out if out is not None else torch.empty((n * cap, 5), dtype=torch.int32, device=dev)
        counts = counts if counts is not None else torch.zeros(n, dtype=torch.int32, device=dev)
        hists = hists if hists is not None else torch.zeros((n, self.nbins_out), dtype=torch.int32, device=dev)
        check(self.lib.dog_detect_batched(self.h, tab.data_ptr(), n, mh, mw, out.data_ptr(), counts.data_ptr(),
                                          hists.data_ptr(), _stream(stream)), "dog_detect_batched")
        return out, counts, hists

    # --------------------------------------------------------- differentiable
    def soft_hist(self, img: torch.Tensor, sigmas: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None, rec: "SoftMaxima | None" = None) -> torch.Tensor:
        """Soft histogram (accumulated into `out`); with `rec`, the maxima are
        recorded for `backward(..., rec=rec)`."""
        H, W, pitch = _check_img(img)
        if out is None:
            out = torch.zeros(self.cfg.nbins, dtype=torch.float32, device=img.device)
        if rec is not None:
            _check_rec(rec, img.device)
        if rec is None:
            check(self.lib.dog_soft_hist(self.h, img.data_ptr(), H, W, pitch, sigmas.data_ptr(), out.data_ptr(),
                                         _stream(stream)), "dog_soft_hist")
        else:
            check(self.lib.dog_soft_hist_rec(self.h, img.data_ptr(), H, W, pitch, sigmas.data_ptr(),
                                             out.data_ptr(), rec.buf.data_ptr(), rec.cap, rec.count.data_ptr(),
                                             _stream(stream)), "dog_soft_hist_rec")
        return out

    def backward(self, img: torch.Tensor, sigmas: torch.Tensor, grad_hist: torch.Tensor,
                 grad_sigmas: torch.Tensor | None = None, stream=None, rec: "SoftMaxima | None" = None):
        """dloss/dI and (accumulated) dloss/dsigma.  With `rec` (a complete
        record of this frame's forward at the same sigmas) the dloss/dL planes
        come from the recorded maxima; otherwise the blur levels are
        recomputed."""
        H, W, pitch = _check_img(img)
        gi = torch.empty((H, W), dtype=torch.float32, device=img.device)
        gs = grad_sigmas if grad_sigmas is not None else torch.zeros(self.K, dtype=torch.float32,
                                                                   device=img.device)
        g = grad_hist.contiguous()
        if rec is not None:
            _check_rec(rec, img.device)
        if rec is None:
            check(self.lib.dog_backward(self.h, img.data_ptr(), H, W, pitch, sigmas.data_ptr(),
                                        g.data_ptr(), gi.data_ptr(), gs.data_ptr(), _stream(stream)), "dog_backward")
        else:
            check(self.lib.dog_backward_rec(self.h, img.data_ptr(), H, W, pitch, sigmas.data_ptr(),
                                            rec.buf.data_ptr(), rec.count.data_ptr(), rec.cap, g.data_ptr(),
                                            gi.data_ptr(), gs.data_ptr(), _stream(stream)), "dog_backward_rec")
        return gi, gs


def blobs_from_raw(raw: torch.Tensor, count: int):
    r = raw[:count].cpu()
    ints = r[:, :3].numpy()
    flt = r[:, 3:].view(torch.float32).numpy()
    return ints[:, 0], ints[:, 1], ints[:, 2], flt[:, 0], flt[:, 1]


def _check_rec(rec: "SoftMaxima", device) -> None:
    if (rec.buf.dtype != torch.int32 or tuple(rec.buf.shape) != (rec.cap, 6) or not rec.buf.is_contiguous()
            or rec.buf.device != device or rec.count.device != device or rec.count.dtype != torch.int32):
        raise ValueError("SoftMaxima: int32 (cap, 6) record and int32 count on the frame's device expected")


class SoftMaxima:
    """Device list of the hard local maxima one soft-histogram forward found
    (`dog_soft_max` records, 24 bytes each) and its true count."""

    def __init__(self, cap: int, device):
        self.cap = int(cap)
        self.buf = torch.empty((self.cap, 6), dtype=torch.int32, device=device)
        self.count = torch.zeros((), dtype=torch.int32, device=device)


class DoGSoftHist(torch.autograd.Function):
    """Soft blob-volume histogram of a batch of frames with learnable sigmas.

    forward(frames (B, H, W) float32 CUDA, sigmas (K,) float32 CUDA, det) ->
    H (nbins,) summed over the batch.  The forward records each frame's hard
    maxima (O(maxima) memory, no blur level is kept); backward scatters the
    dloss/dL planes from them and runs the adjoint blurs.  A frame whose list
    overflowed (more maxima than `rec_cap`, e.g. a flat frame where every
    voxel ties) recomputes its blur levels in the backward instead."""

    rec_cap = 1 << 18

    @staticmethod
    def forward(ctx, frames: torch.Tensor, sigmas: torch.Tensor, det: Detector):
        frames = frames.contiguous()
        sig = sigmas.detach().contiguous()
        out = torch.zeros(det.cfg.nbins, dtype=torch.float32, device=frames.device)
        grads = any(ctx.needs_input_grad[:2])
        recs = [SoftMaxima(DoGSoftHist.rec_cap, frames.device) if grads else None for _ in range(frames.shape[0])]
        for b in range(frames.shape[0]):
            det.soft_hist(frames[b], sig, out=out, rec=recs[b])
        ctx.save_for_backward(frames, sig)
        ctx.det = det
        ctx.recs = recs
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        frames, sig = ctx.saved_tensors
        det = ctx.det
        recs = ctx.recs
        counts = torch.stack([r.count for r in recs]).cpu().tolist()   # one sync per batch
        if any(c > r.cap for c, r in zip(counts, recs)):
            # the overflowed record set the capacity flag; anything else is an error
            st = det.status()
            if st not in (0, _lib.DOG_ERR_CAPACITY):
                check(st, "dog_soft_hist_rec")
        gs = torch.zeros(det.K, dtype=torch.float32, device=frames.device)
        gimg = torch.empty_like(frames)
        g = grad_out.contiguous().float()
        for b in range(frames.shape[0]):
            rec = recs[b] if counts[b] <= recs[b].cap else None
            gi, _ = det.backward(frames[b], sig, g, grad_sigmas=gs, rec=rec)
            gimg[b].copy_(gi)
        return gimg, gs, None
