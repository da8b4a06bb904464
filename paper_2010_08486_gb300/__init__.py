"""GB300-native (sm_103a) Difference-of-Gaussians blob detector.

Implements the data-parallel path of arXiv 2010.08486 (Sec. 3-4): Gaussian
scale space over a sigma ladder, adjacent-scale differences, 3x3x3 local
maxima above a threshold, overlap pruning and the blob-volume histogram,
as hand-written CUDA kernels behind the C ABI in include/dog.h.

Importing this package loads nothing; the CUDA library is loaded on first
use and its absence is an error (there is no CPU fallback).
"""

__all__ = ["Detector", "DetectorConfig", "DoGSoftHist", "small_frame_config", "plif_config",
           "grad_config"]


def __getattr__(name):
    if name in __all__:
        from . import dog
        return getattr(dog, name)
    raise AttributeError(name)
