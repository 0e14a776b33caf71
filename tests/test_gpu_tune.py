"""FFT schedules on the GPU: every z-t tile width and radix order the
autotuner may pick computes the same Fourier acceleration.

- Tile widths only regroup the same line transforms: results are
  bit-identical to the default schedule, after single steps and after a fix.
- The reversed radix order is another exact factorisation, rounded
  differently in FP32: the accelerated gradient matches the oracle within
  the FP32 tolerance of the other parity tests, and a fix to theta < 1e-15
  ends at the oracle's F to 1e-12.
- The pair split (radix order 2: two threads per line, the first radix-2
  stage across the pair) has the stage sequence of the reversed order for
  lines of 8 and 32, and gives bit-identical results there; elsewhere it is
  a third factorisation, checked against the oracle like the reversed order.
- lgf_autotune picks one of them; a cache file written under LGF_TUNE_CACHE
  and loaded back gives new handles of that shape the same schedule.
"""
import ctypes
import os

import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu
ALPHA = 0.08


@pytest.fixture(scope="module")
def lgf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1208_1186_gb300 as P
    from paper_1208_1186_gb300.build import build
    build()
    P._lib.load().lgf_tune_clear()
    yield P
    P._lib.load().lgf_tune_clear()


def run(lgf, dims, dtype, sched, U, n_iter):
    with lgf.GaugeFixer(dims, dtype) as gf:
        if sched is not None:
            gf.set_schedule(*sched)
        gf.load_links(U)
        pr = gf.probe()
        gf.iterate(n_iter)
        out = gf.store_links()
        gf.load_links(U)
        it, conv = gf.fix(1e-15, 2000)
        F, th = gf.functional()
        assert conv and th < 1e-15
        return pr["delta_tilde"], out, it, F, gf.store_links()


@pytest.mark.parametrize("dtype,dims,bx", [("f32", (32, 32, 8, 8), 8), ("f32", (16, 16, 32, 16), 8),
                                           ("f64", (32, 32, 8, 8), 4)])
def test_tile_widths_are_bit_identical(lgf, dtype, dims, bx):
    U = I.synthetic_config(dims, seed=11, link_scale=0.5)
    ref = run(lgf, dims, dtype, None, U, 5)
    got = run(lgf, dims, dtype, (3, bx, 0), U, 5)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert got[2] == ref[2] and got[3] == ref[3] and np.array_equal(got[4], ref[4])


@pytest.mark.parametrize("dims", [(32, 32, 8, 8), (12, 12, 32, 8)])
@pytest.mark.parametrize("bx", [0, 8])
def test_reversed_radix_order_matches_the_oracle(lgf, dims, bx):
    if dims[0] % (bx or 4):
        pytest.skip("tile width does not divide Lx")
    U = I.synthetic_config(dims, seed=12, link_scale=0.5)
    parts = O.step_parts(U, ALPHA)
    Dt_ref = O.pack_delta(parts["Delta_tilde"])
    ref_fix = O.fix(U, 1e-15, 2000, ALPHA)
    dt, _, it, F, _ = run(lgf, dims, "f32", (3, bx, 1), U, 1)
    # FP32 forward + inverse FFT: error ~ eps log2 V of the largest entry
    assert np.max(np.abs(dt - Dt_ref)) <= 4e-6 * np.max(np.abs(Dt_ref))
    assert F == pytest.approx(ref_fix["F"], rel=1e-12)


@pytest.mark.parametrize("bx", [0, 8])
def test_pair_split_equals_the_reversed_order_for_lines_of_32_and_8(lgf, bx):
    dims = (16, 16, 32, 8)
    U = I.synthetic_config(dims, seed=14, link_scale=0.5)
    ref = run(lgf, dims, "f32", (3, bx, 1), U, 5)
    got = run(lgf, dims, "f32", (3, bx, 2), U, 5)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert got[2] == ref[2] and got[3] == ref[3] and np.array_equal(got[4], ref[4])


@pytest.mark.parametrize("bx", [0, 8])
def test_pair_split_matches_the_oracle(lgf, bx):
    dims = (16, 16, 16, 16)
    U = I.synthetic_config(dims, seed=15, link_scale=0.5)
    parts = O.step_parts(U, ALPHA)
    Dt_ref = O.pack_delta(parts["Delta_tilde"])
    ref_fix = O.fix(U, 1e-15, 2000, ALPHA)
    dt, _, it, F, _ = run(lgf, dims, "f32", (3, bx, 2), U, 1)
    assert np.max(np.abs(dt - Dt_ref)) <= 4e-6 * np.max(np.abs(Dt_ref))
    assert F == pytest.approx(ref_fix["F"], rel=1e-12)


def test_autotune_choice_and_cache_file(lgf, tmp_path):
    dims = (32, 32, 8, 8)
    U = I.synthetic_config(dims, seed=13, link_scale=0.5)
    lib = lgf._lib.load()
    path = tmp_path / "tune.json"
    os.environ["LGF_TUNE_CACHE"] = str(path)
    try:
        with lgf.GaugeFixer(dims, "f32") as gf:
            gf.load_links(U)
            gf.autotune(reps=3)
            chosen = gf.schedule()
            gf.load_links(U)
            it, conv = gf.fix(1e-15, 2000)
            F = gf.functional()[0]
    finally:
        del os.environ["LGF_TUNE_CACHE"]
    assert conv
    assert chosen[0] in (1, 2, 3)
    ref = O.fix(U, 1e-15, 2000, ALPHA)
    assert F == pytest.approx(ref["F"], rel=1e-12)
    assert path.exists()
    lib.lgf_tune_clear()
    n = ctypes.c_int(0)
    assert lib.lgf_tune_load(str(path).encode(), ctypes.byref(n)) == 0 and n.value >= 1
    with lgf.GaugeFixer(dims, "f32") as gf:
        assert gf.schedule() == chosen
    lib.lgf_tune_clear()
    with lgf.GaugeFixer(dims, "f32") as gf:
        assert gf.schedule() == (3, 0, 0)  # the default again
