"""The C-ABI library builds, loads without a GPU and exports every function
include/dog.h declares; host-only entry points behave (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2010_08486_gb300 import _lib
from paper_2010_08486_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dog.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dog_[a-z_]+)\s*\(", src, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declarations_listed():
    decl = _declared()
    assert len(decl) == len(set(decl))
    assert tuple(decl) == _lib.EXPORTS


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_entry_points():
    L = _lib.load()
    for code, name in [(0, b"ok"), (-4, b"blob list capacity exceeded"), (-6, b"unsupported configuration")]:
        assert L.dog_status_string(code) == name
    c = _lib.DogConfig()
    assert L.dog_config_default(ctypes.byref(c)) == 0
    assert (c.min_sigma, c.max_sigma, c.ratio, c.threshold, c.overlap, c.nbins) == (1.0, 10.0, 1.6, 0.1, 0.5, 32)
    assert L.dog_config_default(None) == _lib.DOG_ERR_INVALID
    # invalid configs are rejected before any device call
    c.overlap = 1.5
    h = ctypes.c_void_p()
    assert L.dog_create(ctypes.byref(c), ctypes.byref(h)) == _lib.DOG_ERR_INVALID
    assert L.dog_set_tiling(None, 8, 1) == _lib.DOG_ERR_INVALID
    assert L.dog_ring_hist_push(None, 4, None, 4, None, None, None) == _lib.DOG_ERR_INVALID


def test_struct_layouts():
    assert ctypes.sizeof(_lib.DogFrame) == 32
    assert _lib.BLOB_BYTES == 20
