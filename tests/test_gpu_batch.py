"""Batches (lgf_batch_*) and the FFT-pipeline autotuner on the GPU.

A batch runs each member's own kernel chain (the same launches in the same
order as a single handle) from one CUDA graph per host check, so a batched
fix must reproduce every member's individual fix exactly: the same number
of updates and bit-identical links."""
import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu

MEMBERS = [((8, 8, 8, 8), "f64", 0), ((12, 12, 32, 8), "f32", 1), ((6, 12, 4, 20), "f32_r12", 2),
           ((4, 6, 10, 12), "f64_r12", 3), ((8, 8, 32, 16), "f32", 4)]


@pytest.fixture(scope="module")
def lgf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1208_1186_gb300 as P
    from paper_1208_1186_gb300.build import build
    build()
    return P


def _inputs():
    return [I.synthetic_config(d, seed=s, link_scale=0.5) for d, _, s in MEMBERS]


@pytest.mark.parametrize("lanes", [None, 1, 2])
def test_batch_fix_reproduces_individual_fixes(lgf, lanes):
    """Lanes change only how members' kernel chains share the GPU, never a
    member's own arithmetic."""
    Us = _inputs()
    singles = []
    for (d, dt, _), U in zip(MEMBERS, Us):
        with lgf.GaugeFixer(d, dt) as gf:
            gf.load_links(U)
            it, conv = gf.fix(1e-15, 2000)
            singles.append((it, conv, gf.fix_split(), gf.store_links(), gf.functional()))
    fixers = [lgf.GaugeFixer(d, dt) for d, dt, _ in MEMBERS]
    try:
        for f, U in zip(fixers, Us):
            f.load_links(U)
        with lgf.GaugeBatch(fixers) as b:
            if lanes is not None:
                b.set_lanes(lanes)
            its, convs = b.fix(1e-15, 2000)
        for k, f in enumerate(fixers):
            it, conv, split, links, (F, th) = singles[k]
            assert its[k] == it and convs[k] == conv, MEMBERS[k]
            assert f.fix_split() == split
            assert np.array_equal(f.store_links(), links), MEMBERS[k]
            assert f.functional() == (F, th)
            assert conv and th < 1e-15
    finally:
        for f in fixers:
            f.close()


def test_batch_iterate_reproduces_individual_iterations(lgf):
    Us = _inputs()
    fixers = [lgf.GaugeFixer(d, dt) for d, dt, _ in MEMBERS]
    try:
        for f, U in zip(fixers, Us):
            f.load_links(U)
        with lgf.GaugeBatch(fixers) as b:
            b.iterate(7)
            b.iterate(0)
        for (d, dt, _), U, f in zip(MEMBERS, Us, fixers):
            with lgf.GaugeFixer(d, dt) as gf:
                gf.load_links(U)
                gf.iterate(7)
                assert np.array_equal(gf.store_links(), f.store_links()), d
    finally:
        for f in fixers:
            f.close()


def test_batch_rejects_duplicates_and_unloaded(lgf):
    with lgf.GaugeFixer((4, 4, 4, 4), "f64") as a, lgf.GaugeFixer((4, 4, 4, 6), "f64") as c:
        with pytest.raises(lgf.LgfError, match="twice"):
            lgf.GaugeBatch([a, a])
        with lgf.GaugeBatch([a, c]) as b:
            with pytest.raises(lgf.LgfError, match="no links loaded"):
                b.fix(1e-12, 10)


@pytest.mark.parametrize("dims,dtype", [((8, 8, 8, 8), "f64"), ((12, 12, 32, 8), "f32"), ((6, 12, 4, 20), "f32")])
def test_autotune_picks_an_available_pipeline(lgf, dims, dtype):
    U = I.synthetic_config(dims, seed=3, link_scale=0.5)
    ref = O.fix(U, 1e-14, 2000, 0.08)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        chosen = gf.autotune(reps=3)
        assert chosen in (1, 2, 3)
        assert np.array_equal(gf.store_links(), gf.store_links())
        it, conv = gf.fix(1e-14, 2000)
        F, th = gf.functional()
    assert conv and th < 1e-14
    assert F == pytest.approx(ref["F"], rel=1e-12)


def test_batch_lane_autotuner_keeps_results(lgf):
    """The lane autotuner returns one of its candidates; a fix after it (from
    freshly loaded links) still reproduces the individual fixes."""
    Us = _inputs()
    singles = []
    for (d, dt, _), U in zip(MEMBERS, Us):
        with lgf.GaugeFixer(d, dt) as gf:
            gf.load_links(U)
            gf.fix(1e-15, 2000)
            singles.append(gf.store_links())
    fixers = [lgf.GaugeFixer(d, dt) for d, dt, _ in MEMBERS]
    try:
        for f, U in zip(fixers, Us):
            f.load_links(U)
        with lgf.GaugeBatch(fixers) as b:
            lanes = b.autotune(reps=2)
            assert lanes in (0, 1, 2, 4)  # candidates up to the member count (5)
            for f, U in zip(fixers, Us):
                f.load_links(U)
            b.fix(1e-15, 2000)
        for k, f in enumerate(fixers):
            assert np.array_equal(f.store_links(), singles[k]), MEMBERS[k]
    finally:
        for f in fixers:
            f.close()
