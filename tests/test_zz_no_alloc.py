"""lgf_functional_noalloc: F and theta without any device allocation.

This entry point serves callers that may not allocate GPU memory (a host
program that keeps the device memory in its own pool and forbids its
libraries to call cudaMalloc, or a monitor that must not change the memory
footprint of the job it watches).  The links and the output live in memory
the caller already owns; the library's only scratch is a fixed array compiled
into it.  The GPU test checks two calls in a row, on different lattices,
against lgf_functional, the entry point that allocates its own buffers, and
against the FP64 oracle's F and theta of the same links.  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O
from paper_1208_1186_gb300 import _lib
from paper_1208_1186_gb300.build import build

NC = {"f64": 9, "f64_r12": 6, "f32": 9, "f32_r12": 6}


def soa_links(U, dtype):
    """Host links -> the library's device storage: [mu][c][s] complex planes."""
    import torch
    V = U.size // 36
    a = U.reshape(V, 4, 9)[:, :, :NC[dtype]]
    a = np.ascontiguousarray(a.transpose(1, 2, 0))
    a = a.astype(np.complex128 if dtype.startswith("f64") else np.complex64)
    return torch.from_numpy(a).to("cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32", "f64_r12", "f32_r12"])
def test_noalloc_functional_matches_lgf_functional(dtype):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    import paper_1208_1186_gb300 as lgf
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    # two calls in a row: the second lattice uses fewer block sums than the first
    for dims, seed in [((8, 8, 12, 16), 1), ((4, 6, 10, 2), 2)]:
        U = I.synthetic_config(dims, seed=seed, link_scale=0.5)
        with lgf.GaugeFixer(dims, dtype) as gf:
            gf.load_links(U)
            F_ref, th_ref = gf.functional()
        links = soa_links(U, dtype)
        torch.cuda.synchronize()
        st = lib.lgf_functional_noalloc(ctypes.c_void_p(links.data_ptr()), *dims, _lib.DTYPES[dtype],
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == _lib.LGF_OK, lib.lgf_last_error(None)
        torch.cuda.synchronize()
        F, th = out.tolist()
        # FP64 storage: both sides sum FP64 terms (rel 1e-13 / 1e-12, as in
        # the FP64 parity tests).  FP32 storage: lgf_functional sums each warp
        # in FP32 before the FP64 sum, this entry point sums FP64 terms, so
        # they agree to FP32 rounding (rel 1e-6 / 1e-5, as the FP32 tests).
        rel_F, rel_th = (1e-13, 1e-12) if dtype.startswith("f64") else (1e-6, 1e-5)
        assert F == pytest.approx(F_ref, rel=rel_F)
        assert th == pytest.approx(th_ref, rel=rel_th)
        # the oracle's FP64 F and theta of the unrounded links: FP32 storage
        # rounds each entry by 2^-24 relative, which moves F and theta by
        # about that much relative (theta of these links is O(1))
        F_o, th_o = O.functional(U)
        assert F == pytest.approx(F_o, rel=rel_F)
        assert th == pytest.approx(th_o, rel=rel_th)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    """Host-side check, before any device work: 64^3 x 20 sites > 4,194,304."""
    build()
    lib = _lib.load()
    st = lib.lgf_functional_noalloc(None, 64, 64, 64, 20, _lib.LGF_F64, None, None)
    assert st == _lib.LGF_ERR_ARG
    assert b"at most 4194304" in lib.lgf_last_error(None)
