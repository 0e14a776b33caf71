"""The gauge step with the exact exponential (LGF_EXP_ORDER = 0) on the GPU,
against the oracle's exp_order = 0 (g = reunitarised exp(alpha/2 Delta~), the
exponential by eigen-decomposition, itself pinned against scipy's expm in
test_oracle.py).

The library forms the exponential by a Taylor series with scaling and
squaring (degree 16 in FP64): its truncation error (~2e-20) and rounding
(~1e-16 of |g| = 1) sit far below the 1e-12 that the FP64 steps are held to,
as the first-order steps are in test_gpu_parity.py.  The FP32 storage path is
judged by its FP64-tail result, the final F to 1e-12 relative."""
import functools

import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu

ALPHA = 0.08
LGF_EXP_ORDER = 8


@pytest.fixture(scope="module")
def lgf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1208_1186_gb300 as P
    from paper_1208_1186_gb300.build import build
    build()
    return P


@pytest.mark.parametrize("dtype", ["f64", "f64_r12"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 12, 4, 20), (4, 6, 10, 12), (2, 2, 2, 2)])
def test_exact_exp_step_matches_oracle(lgf, dims, dtype):
    U = I.synthetic_config(dims, seed=3, link_scale=0.5)
    ref = O.step_parts(U, ALPHA, exp_order=0)
    first = O.step_parts(U, ALPHA, exp_order=1)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.set_param(LGF_EXP_ORDER, 0)
        gf.load_links(U)
        out = gf.probe()
        gf.iterate(1)
        U1 = gf.store_links()
    np.testing.assert_allclose(out["g"], ref["g"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(U1, ref["U_next"], rtol=0, atol=1e-12)
    # the two orders differ by far more than the tolerance: the test sees which one ran
    assert np.max(np.abs(ref["g"] - first["g"])) > 1e-6


def test_exact_exp_iterations_and_fix_match_oracle(lgf):
    """8^4 FP64 (link scale 0.3, seed 0): links after 50 exact-exponential
    iterations to 1e-10, and lgf_fix's update count and theta history."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=0, link_scale=0.3)
    ref50 = O.iterate(U, 50, ALPHA, exp_order=0)
    ref = O.fix(U, 1e-12, 2000, ALPHA, exp_order=0)
    with lgf.GaugeFixer(dims, "f64") as gf:
        gf.set_param(LGF_EXP_ORDER, 0)
        gf.load_links(U)
        gf.iterate(50)
        assert np.max(np.abs(gf.store_links() - ref50)) <= 1e-10
        gf.load_links(U)
        iters, conv = gf.fix(1e-12, 2000)
        F, th = gf.functional()
        hist = gf.history()
        out = gf.store_links()
    assert conv and ref["converged"]
    assert iters == ref["iterations"]
    assert F == pytest.approx(ref["F"], rel=1e-13)
    np.testing.assert_allclose(hist, [h[1] for h in ref["history"]], rtol=1e-9, atol=1e-25)
    assert np.max(np.abs(out - ref["U"])) <= 1e-10


@functools.lru_cache(maxsize=None)
def _oracle_fix_exact(dims):
    U = I.synthetic_config(dims, seed=2, link_scale=0.5)
    return U, O.fix(U, 1e-15, 2000, ALPHA, exp_order=0)


@pytest.mark.parametrize("reunit_fp64", [0, 1])
@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 10, 12)])
def test_exact_exp_mixed_precision_fix(lgf, dims, dtype, reunit_fp64):
    U, ref = _oracle_fix_exact(dims)
    assert ref["converged"]
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.set_param(LGF_EXP_ORDER, 0)
        gf.set_param(4, reunit_fp64)  # LGF_REUNIT_FP64
        gf.load_links(U)
        iters, conv = gf.fix(1e-15, 2000)
        F, th = gf.functional()
        out = gf.store_links()
    assert conv and th < 1e-15
    assert F == pytest.approx(ref["F"], rel=1e-12)
    assert O.unitarity_defect(out) < 1e-12
    assert O.average_plaquette(out) == pytest.approx(O.average_plaquette(U), abs=1e-12)


def test_exp_order_rejects_other_values(lgf):
    with lgf.GaugeFixer((4, 4, 4, 4), "f64") as gf:
        for bad in (2, -1, 0.5):
            with pytest.raises(lgf.LgfError):
                gf.set_param(LGF_EXP_ORDER, bad)
        gf.set_param(LGF_EXP_ORDER, 1)
