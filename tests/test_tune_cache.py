"""The FFT schedule cache of the autotuner as a JSON file, on the host (no
GPU): lgf_tune_load takes the valid entries of a file into the process
cache, lgf_tune_lookup reads them back, lgf_tune_save writes a file that is
valid JSON and loads back to the same cache, and entries no engine could run
(a tile width that does not divide Lx, a radix order where the stages would
not change or in FP64, a pair split without kernels for the lattice, a
pipeline the lattice does not support) are rejected."""
import ctypes
import json

import pytest

from paper_1208_1186_gb300 import _lib
from paper_1208_1186_gb300.build import build

VALID = [
    (4, (32, 32, 32, 32), 3, 8, 1),   # FP32 register planes, 8-wide z-t tiles, reversed radix order
    (4, (48, 48, 48, 8), 3, 4, 0),
    (8, (32, 32, 32, 32), 3, 4, 0),   # FP64: widths 2 (default, 0) and 4
    (4, (16, 16, 16, 16), 2, 0, 0),   # per-axis passes
    (8, (10, 4, 6, 12), 1, 0, 0),     # Stockham planes
    (4, (24, 24, 24, 24), 3, 0, 2),   # pair-split z and t transforms
]
INVALID = [
    (4, (20, 20, 20, 20), 3, 8, 0),   # 8 does not divide Lx = 20
    (4, (16, 16, 16, 16), 3, 0, 1),   # radix order 1 changes no stage of 16
    (8, (32, 32, 32, 32), 3, 4, 1),   # FP64 runs radix order 0 only
    (4, (10, 10, 10, 10), 3, 0, 0),   # no register-plane kernels for 10
    (4, (32, 32, 32, 32), 2, 4, 0),   # a tile width outside the plane pipeline
    (2, (32, 32, 32, 32), 1, 0, 0),   # no 2-byte precision
    (4, (32, 32, 32, 70), 1, 0, 0),   # extent beyond 64
    (4, (8, 8, 8, 8), 3, 0, 2),       # no pair-split kernels for lines this short
    (8, (16, 16, 16, 16), 3, 0, 2),   # the pair split is FP32 only
]


@pytest.fixture()
def lib():
    build()
    lib = _lib.load()
    lib.lgf_tune_clear()
    yield lib
    lib.lgf_tune_clear()


def entry_line(prec, L, p, b, r, ms=0.05):
    return (f' {{"prec": {prec}, "L": [{L[0]}, {L[1]}, {L[2]}, {L[3]}], "pipeline": {p}, "zt_bx": {b}, '
            f'"zt_ro": {r}, "ms": {ms}}}')


def lookup(lib, prec, L):
    p, b, r = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int(-1)
    st = lib.lgf_tune_lookup(prec, *L, ctypes.byref(p), ctypes.byref(b), ctypes.byref(r))
    return st, (p.value, b.value, r.value)


def test_load_lookup_save_round_trip(lib, tmp_path):
    src = tmp_path / "in.json"
    lines = [entry_line(*e) for e in VALID + INVALID]
    src.write_text('{"lgf_fft_schedules": [\n' + ",\n".join(lines) + "\n]}\n")
    n = ctypes.c_int(0)
    assert lib.lgf_tune_load(str(src).encode(), ctypes.byref(n)) == _lib.LGF_OK
    assert n.value == len(VALID)
    for prec, L, p, b, r in VALID:
        assert lookup(lib, prec, L) == (_lib.LGF_OK, (p, b, r))
    for prec, L, *_ in INVALID:
        if (prec, L) not in [(v[0], v[1]) for v in VALID]:
            assert lookup(lib, prec, L)[0] == _lib.LGF_ERR_ARG
    out = tmp_path / "out.json"
    assert lib.lgf_tune_save(str(out).encode()) == _lib.LGF_OK
    data = json.loads(out.read_text())
    got = {(e["prec"], tuple(e["L"])): (e["pipeline"], e["zt_bx"], e["zt_ro"]) for e in data["lgf_fft_schedules"]}
    assert got == {(prec, L): (p, b, r) for prec, L, p, b, r in VALID}
    assert all(abs(e["ms"] - 0.05) < 1e-9 for e in data["lgf_fft_schedules"])
    # cleared, then loaded back from the saved file: the same cache
    lib.lgf_tune_clear()
    assert lookup(lib, *VALID[0][:2])[0] == _lib.LGF_ERR_ARG
    assert lib.lgf_tune_load(str(out).encode(), ctypes.byref(n)) == _lib.LGF_OK and n.value == len(VALID)
    for prec, L, p, b, r in VALID:
        assert lookup(lib, prec, L) == (_lib.LGF_OK, (p, b, r))


def test_missing_file_is_an_argument_error(lib, tmp_path):
    assert lib.lgf_tune_load(str(tmp_path / "none.json").encode(), None) == _lib.LGF_ERR_ARG
    assert b"cannot read" in lib.lgf_last_error(None)
    assert lib.lgf_tune_save(str(tmp_path / "no_dir" / "x.json").encode()) == _lib.LGF_ERR_ARG
