"""ctypes binding of libdog.so (include/dog.h).  Argument marshalling only.

Loading fails loudly: there is no CPU or Python fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdog.so")

DOG_OK = 0
DOG_ERR_INVALID = -1
DOG_ERR_NOMEM = -2
DOG_ERR_CUDA = -3
DOG_ERR_CAPACITY = -4
DOG_ERR_TIMEOUT = -5
DOG_ERR_UNSUPPORTED = -6

LADDER_GEOM, LADDER_ARITH = 0, 1
NORM_DERIV, NORM_PAPER = 0, 1
PRUNE_COALESCE, PRUNE_SUPPRESS, PRUNE_OFF = 0, 1, 2
HIST_LOGV, HIST_LADDER = 0, 1
DTYPE_F32, DTYPE_U16 = 0, 1
BACKEND_DIRECT, BACKEND_FFT = 0, 1
MAX_LEVELS = 32
MAX_RADIUS = 64
NOALLOC_MAX_CAND = 65536

# Every function declared in include/dog.h, in declaration order.
EXPORTS = (
    "dog_config_default", "dog_create", "dog_destroy", "dog_ladder", "dog_candidates", "dog_prune",
    "dog_prune_noalloc", "dog_stretch_limits", "dog_stretch", "dog_render_spheres", "dog_volume_hist", "dog_detect", "dog_detect_batched", "dog_set_tiling", "dog_set_producer_warps", "dog_get_producer_warps", "dog_soft_hist",
    "dog_backward", "dog_soft_hist_rec", "dog_backward_rec", "dog_debug_dog", "dog_ring_hist_push", "dog_ring_hist_push_batched",
    "dog_profile_enable", "dog_profile_read", "dog_fma_peak",
    "dog_get_status", "dog_test_fail_alloc", "dog_status_string",
)


class DogConfig(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int32),
        ("sigmas", ctypes.POINTER(ctypes.c_double)),
        ("min_sigma", ctypes.c_double),
        ("max_sigma", ctypes.c_double),
        ("ratio", ctypes.c_double),
        ("ladder", ctypes.c_int32),
        ("truncate", ctypes.c_double),
        ("threshold", ctypes.c_double),
        ("overlap", ctypes.c_double),
        ("norm", ctypes.c_int32),
        ("prune", ctypes.c_int32),
        ("nbins", ctypes.c_int32),
        ("hist_mode", ctypes.c_int32),
        ("soft_T", ctypes.c_double),
        ("max_h", ctypes.c_int32),
        ("max_w", ctypes.c_int32),
        ("blob_cap", ctypes.c_int32),
        ("stretch_sat", ctypes.c_double),
        ("backend", ctypes.c_int32),
    ]


class DogFrame(ctypes.Structure):
    _fields_ = [
        ("ptr", ctypes.c_void_p),
        ("h", ctypes.c_int32),
        ("w", ctypes.c_int32),
        ("pitch", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("blob_off", ctypes.c_int64),
    ]


BLOB_BYTES = 20
FRAME_BYTES = ctypes.sizeof(DogFrame)

_lock = threading.Lock()
_lib = None


class DogError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        name = "unknown"
        try:
            name = load().dog_status_string(code).decode()
        except Exception:
            pass
        super().__init__("%s failed: %s (%d)" % (where, name, code))


def check(code: int, where: str) -> None:
    if code != DOG_OK:
        raise DogError(code, where)


def load(path: str | None = None):
    """Load libdog.so; raises if it is missing (build it with build.py)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("DOG_LIB", LIB_PATH)
        if not os.path.exists(p):
            raise RuntimeError("libdog.so not found at %s: build it with "
                               "`python -m paper_2010_08486_gb300.build`" % p)
        lib = ctypes.CDLL(p)
        vp, i32, P = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER
        lib.dog_config_default.argtypes = [P(DogConfig)]
        lib.dog_create.argtypes = [P(DogConfig), P(vp)]
        lib.dog_destroy.argtypes = [vp]
        lib.dog_destroy.restype = None
        lib.dog_ladder.argtypes = [vp, P(i32), P(ctypes.c_double), P(i32), P(ctypes.c_double)]
        lib.dog_candidates.argtypes = [vp, vp, i32, i32, i32, i32, vp, i32, vp, vp]
        lib.dog_prune.argtypes = [vp, vp, vp, i32, i32, i32, vp, i32, vp, vp]
        lib.dog_prune_noalloc.argtypes = [vp, vp, i32, P(ctypes.c_double), i32, ctypes.c_double, i32, vp, i32,
                                          vp, vp]
        lib.dog_stretch_limits.argtypes = [vp, i32, i32, i32, ctypes.c_double, vp, vp, vp]
        lib.dog_stretch.argtypes = [vp, i32, i32, i32, vp, vp, i32, vp]
        lib.dog_render_spheres.argtypes = [vp, i32, i32, i32, i32, ctypes.c_float, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_uint64, vp, vp, i32, vp]
        lib.dog_volume_hist.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        lib.dog_detect.argtypes = [vp, vp, i32, i32, i32, i32, vp, i32, vp, vp, vp, vp]
        lib.dog_detect_batched.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp]
        lib.dog_set_tiling.argtypes = [vp, i32, i32]
        lib.dog_set_producer_warps.argtypes = [vp, i32]
        lib.dog_get_producer_warps.argtypes = [vp]
        lib.dog_soft_hist.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp]
        lib.dog_backward.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
        lib.dog_soft_hist_rec.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, i32, vp, vp]
        lib.dog_backward_rec.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, i32, vp, vp, vp, vp]
        lib.dog_debug_dog.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp]
        lib.dog_ring_hist_push.argtypes = [vp, i32, vp, i32, vp, vp, vp]
        lib.dog_ring_hist_push_batched.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, vp, vp]
        lib.dog_profile_enable.argtypes = [vp, i32]
        lib.dog_profile_read.argtypes = [vp, P(ctypes.c_double), P(i32)]
        lib.dog_fma_peak.argtypes = [i32, ctypes.c_int64, i32, P(ctypes.c_double), P(ctypes.c_double), vp]
        lib.dog_get_status.argtypes = [vp, P(i32)]
        lib.dog_test_fail_alloc.argtypes = [i32]
        lib.dog_status_string.argtypes = [ctypes.c_int]
        lib.dog_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("dog_destroy", "dog_status_string"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib
