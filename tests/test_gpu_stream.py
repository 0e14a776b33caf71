"""Streamed fixing of an ensemble (lgf_fix_stream) on the GPU.

The streaming executor only changes where the host copies run (device
staging buffers on copy streams of their own, overlapping the fixing of the
neighbouring configurations); every configuration still runs the handle's
own load, fix and store kernels in the same order.  So each streamed result
must equal the plain lgf_load_links + lgf_fix + lgf_store_links sequence bit
for bit, with the same update count, and the fixed links must satisfy the
Landau condition as the oracle recomputes it."""
import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1208_1186_gb300 as P
    from paper_1208_1186_gb300.build import build
    build()
    return P, torch


def _pinned(torch, shape):
    t = torch.empty(tuple(shape) + (2,), dtype=torch.float64, pin_memory=True)
    return t, t.numpy().view(np.complex128).reshape(shape)


def _sequential(P, dims, dt, Us, tol, max_iter):
    out = []
    with P.GaugeFixer(dims, dt) as gf:
        for U in Us:
            gf.load_links(U)
            it, conv = gf.fix(tol, max_iter)
            out.append((it, conv, gf.store_links()))
    return out


@pytest.mark.parametrize("dims,dt,n", [((8, 8, 8, 12), "f32", 5), ((6, 8, 4, 10), "f64", 4),
                                       ((8, 8, 12, 8), "f32_r12", 3)])
def test_stream_matches_sequential_fixes(env, dims, dt, n):
    P, torch = env
    Us = [I.synthetic_config(dims, seed=s, link_scale=0.5) for s in range(n)]
    ref = _sequential(P, dims, dt, Us, 1e-15, 2000)
    keep = []  # the pinned tensors behind the numpy views
    ins, outs = [], []
    for U in Us:
        t, a = _pinned(torch, U.shape)
        a[...] = U
        keep.append(t)
        ins.append(a)
        t, a = _pinned(torch, U.shape)
        a[...] = np.nan  # every output must be written
        keep.append(t)
        outs.append(a)
    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
    with P.GaugeFixer(dims, dt, stream=s0) as f0, P.GaugeFixer(dims, dt, stream=s1) as f1:
        its, conv = P.fix_stream((f0, f1), ins, outs, 1e-15, 2000)
    assert conv
    for k in range(n):
        it, c, links = ref[k]
        assert c and its[k] == it, k
        assert np.array_equal(outs[k], links), k
    # the Landau condition on the streamed links, from the FP64 oracle
    for k in (0, n - 1):
        F, theta = O.functional(outs[k])
        assert theta < 1e-14, (k, theta)


def test_stream_pageable_buffers_and_short_runs(env):
    """Pageable host arrays (synchronous copies), n = 1 (one handle used),
    n = 0, and a max_iter too small to converge: every configuration is still
    stored as far as it got, equal to the sequential fix with that max_iter."""
    P, _ = env
    dims, dt = (8, 8, 8, 8), "f32"
    Us = [I.synthetic_config(dims, seed=10 + s, link_scale=0.5) for s in range(3)]
    with P.GaugeFixer(dims, dt) as f0, P.GaugeFixer(dims, dt) as f1:
        outs = [np.full_like(U, np.nan) for U in Us]
        its, conv = P.fix_stream((f0, f1), Us, outs, 1e-15, 4)
        assert not conv and its == [4, 4, 4]
        for (it, c, links), o in zip(_sequential(P, dims, dt, Us, 1e-15, 4), outs):
            assert it == 4 and not c
            assert np.array_equal(o, links)
        one = [np.full_like(Us[0], np.nan)]
        its, conv = P.fix_stream((f0, f1), Us[:1], one, 1e-15, 2000)
        ref = _sequential(P, dims, dt, Us[:1], 1e-15, 2000)[0]
        assert conv and its == [ref[0]] and np.array_equal(one[0], ref[2])
        assert P.fix_stream((f0, f1), [], [], 1e-15, 10) == ([], True)


def test_stream_rejects_mismatched_handles(env):
    P, _ = env
    U = I.synthetic_config((8, 8, 8, 8), seed=0, link_scale=0.5)
    out = np.empty_like(U)
    with P.GaugeFixer((8, 8, 8, 8), "f32") as f0, P.GaugeFixer((8, 8, 8, 8), "f64") as f1, \
            P.GaugeFixer((8, 8, 8, 12), "f32") as f2:
        for pair in ((f0, f1), (f0, f2), (f0, f0)):
            with pytest.raises(P.LgfError):
                P.fix_stream(pair, [U], [out], 1e-15, 10)
