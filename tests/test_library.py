"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point include/lgf.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1208_1186_gb300 import _lib
from paper_1208_1186_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lgf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(lgf_[a-z_0-9]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_documented_entry_points():
    names = declared_symbols()
    for core in ["lgf_create", "lgf_load_links", "lgf_iterate", "lgf_fix", "lgf_functional"]:
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows the signature of each
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


@pytest.mark.parametrize("dims", [(7, 8, 8, 8), (8, 8, 8, 1), (8, 128, 8, 8), (8, 8, 0, 8), (11, 8, 8, 8)])
def test_create_rejects_unsupported_extents(lib, dims):
    h = ctypes.c_void_p()
    st = lib.lgf_create(*dims, _lib.LGF_F64, ctypes.byref(h))
    assert st == _lib.LGF_ERR_ARG
    assert not h.value
    assert b"extent" in lib.lgf_last_error(None)


def test_create_rejects_unknown_dtype(lib):
    h = ctypes.c_void_p()
    assert lib.lgf_create(8, 8, 8, 8, 9, ctypes.byref(h)) == _lib.LGF_ERR_ARG
    assert b"dtype" in lib.lgf_last_error(None)


def test_null_handles_are_rejected(lib):
    assert lib.lgf_destroy(None) == _lib.LGF_ERR_ARG
    assert lib.lgf_iterate(None, 1) == _lib.LGF_ERR_ARG
    assert lib.lgf_fix(None, 1e-12, 10, None) == _lib.LGF_ERR_ARG
    assert lib.lgf_functional(None, None, None) == _lib.LGF_ERR_ARG
    assert lib.lgf_set_param(None, _lib.LGF_ALPHA, 0.08) == _lib.LGF_ERR_ARG
    assert lib.lgf_launch_count(None) == -1


def test_allocator_hooks_must_come_in_pairs(lib):
    alloc = _lib.ALLOC_FN(lambda n, d, s, u: None)
    assert lib.lgf_set_allocator(alloc, _lib.FREE_FN(), None) == _lib.LGF_ERR_ARG
    assert lib.lgf_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None) == _lib.LGF_OK


def test_package_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="liblgf.so not found"):
        _lib._lib_saved = _lib._lib
        try:
            _lib._lib = None
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = _lib._lib_saved
