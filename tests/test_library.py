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


def test_every_handle_taking_entry_point_rejects_null(lib):
    """Each call that takes a handle, batch or network checks it (and its
    other arguments) before any device work: LGF_ERR_ARG, no crash."""
    E = _lib.LGF_ERR_ARG
    i = ctypes.c_int(0)
    buf = (ctypes.c_double * 8)()
    calls = {
        "lgf_set_stream": (None, None),
        "lgf_load_links": (None, buf),
        "lgf_load_links_device": (None, buf),
        "lgf_store_links": (None, buf),
        "lgf_store_gauge": (None, buf),
        "lgf_fix_stream": (None, None, 2, None, None, 1e-12, 10, None),
        "lgf_probe": (None, None, None, None),
        "lgf_fix_split": (None, ctypes.byref(i), ctypes.byref(i)),
        "lgf_autotune": (None, 3, None),
        "lgf_tune_schedule": (None, 1, None, None, None),
        "lgf_set_schedule": (None, 1, 3, 0, 0),
        "lgf_history": (None, buf, 8, ctypes.byref(i)),
        "lgf_profile": (None, 1),
        "lgf_batch_destroy": (None,),
        "lgf_batch_iterate": (None, 1),
        "lgf_batch_fix": (None, 1e-12, 10, None, None),
        "lgf_batch_autotune": (None, 3, None),
        "lgf_batch_set_lanes": (None, 2),
        "lgf_net_destroy": (None,),
        "lgf_net_get_params": (None, buf),
        "lgf_net_set_params": (None, buf),
        "lgf_net_set_wait_budget": (None, 0),
        "lgf_net_forward": (None, None, None),
        "lgf_net_train_step": (None, None, 0.0, None, None),
        "lgf_net_warm_start": (None, None),
        "lgf_net_conv": (None, 1, 0, None, None, None, None, 8, 8, 8, 8, None),
        "lgf_tune_load": (None, None),
        "lgf_tune_save": (None,),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == E, name
    # bad values with no handle needed
    h = ctypes.c_void_p()
    assert lib.lgf_create(8, 8, 8, 8, _lib.LGF_F64, None) == E
    b = ctypes.c_void_p()
    assert lib.lgf_batch_create(None, 1, ctypes.byref(b)) == E and not b.value
    assert lib.lgf_batch_create(None, 1, None) == E
    assert lib.lgf_net_create(ctypes.c_ulonglong(0), None) == E
    out = (ctypes.c_double * 2)()
    for dims, dt, links, o in [((1, 8, 8, 8), 0, buf, out), ((8, 8, 8, 65), 0, buf, out), ((8, 8, 8, 8), 7, buf, out),
                               ((8, 8, 8, 8), 0, None, out), ((8, 8, 8, 8), 0, buf, None),
                               ((64, 64, 64, 64), 0, buf, out)]:
        assert lib.lgf_functional_noalloc(links, *dims, dt, o, None) == E, dims
    assert not h.value


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
