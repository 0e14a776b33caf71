"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances.  The FP64 path computes the same sums as the oracle in another
order, so each step agrees to a few ulp of the largest term (|U| = 1,
|Delta| <= 8): 1e-12 for the gradient, the accelerated gradient and g.  After
N iterations the links must agree to 1e-10 max-abs per element (the iteration
contracts towards its fixed point, so rounding differences do not grow).  The
FP32 storage path is compared through its FP64-tail result: the final F to
1e-12 relative, theta < 1e-15.
"""
import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu

ALPHA = 0.08

STEP_DIMS = [
    (8, 8, 8, 8),      # C1 shape
    (4, 6, 10, 12),    # radices 2, 3, 5; V = 2880, ragged last block
    (12, 2, 20, 3),    # odd t extent
    (5, 4, 3, 2),      # odd x extent (one x per z-t tile)
    (64, 2, 2, 2),     # longest x
    (2, 2, 2, 64),     # longest t
    (2, 2, 2, 2),      # smallest
]


@pytest.fixture(scope="module")
def lgf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1208_1186_gb300 as P
    from paper_1208_1186_gb300.build import build
    build()
    return P


def _packed(D):
    return O.pack_delta(D)


@pytest.mark.parametrize("dtype", ["f64", "f64_r12"])
@pytest.mark.parametrize("dims", STEP_DIMS)
def test_one_step_matches_oracle(lgf, dims, dtype):
    U = I.synthetic_config(dims, seed=3, link_scale=0.5)
    ref = O.step_parts(U, ALPHA)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        out = gf.probe()
        F, th = gf.functional()
        gf.iterate(1)
        U1 = gf.store_links()
    np.testing.assert_allclose(out["delta"], _packed(ref["Delta"]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["delta_tilde"], _packed(ref["Delta_tilde"]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["g"], ref["g"], rtol=0, atol=1e-12)
    assert F == pytest.approx(ref["F"], rel=1e-13)
    assert th == pytest.approx(ref["theta"], rel=1e-12)
    np.testing.assert_allclose(U1, ref["U_next"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [10, 50, 200])
def test_iterate_matches_oracle_c1(lgf, n):
    """8^4 FP64, links scale 0.3 behind a gauge of scale 1.0, seed 0."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=0, link_scale=0.3, gauge_scale=1.0)
    ref = O.iterate(U, n, ALPHA)
    with lgf.GaugeFixer(dims, "f64") as gf:
        gf.load_links(U)
        gf.iterate(n)
        out = gf.store_links()
    assert np.max(np.abs(out - ref)) <= 1e-10


def test_iterate_r12_matches_oracle(lgf):
    dims = (4, 6, 10, 12)
    U = I.synthetic_config(dims, seed=1, link_scale=0.5)
    ref = O.iterate(U, 30, ALPHA)
    with lgf.GaugeFixer(dims, "f64_r12") as gf:
        gf.load_links(U)
        gf.iterate(30)
        out = gf.store_links()
    assert np.max(np.abs(out - ref)) <= 1e-10


def test_fix_matches_oracle_c1(lgf):
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=0, link_scale=0.3)
    ref = O.fix(U, 1e-12, 2000, ALPHA)
    with lgf.GaugeFixer(dims, "f64") as gf:
        gf.load_links(U)
        iters, conv = gf.fix(1e-12, 2000)
        F, th = gf.functional()
        hist = gf.history()
        out = gf.store_links()
    assert conv and ref["converged"]
    assert iters == ref["iterations"]
    assert th < 1e-12
    assert F == pytest.approx(ref["F"], rel=1e-13)
    np.testing.assert_allclose(hist, [h[1] for h in ref["history"]], rtol=1e-9, atol=1e-25)
    assert np.max(np.abs(out - ref["U"])) <= 1e-10


@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 10, 12)])
def test_mixed_precision_fix_matches_fp64_functional(lgf, dims, dtype):
    U = I.synthetic_config(dims, seed=2, link_scale=0.5)
    ref = O.fix(U, 1e-15, 2000, ALPHA)
    assert ref["converged"]
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        iters, conv = gf.fix(1e-15, 2000)
        F, th = gf.functional()
        out = gf.store_links()
    assert conv and th < 1e-15
    assert F == pytest.approx(ref["F"], rel=1e-12)
    assert O.unitarity_defect(out) < 1e-12
    assert O.average_plaquette(out) == pytest.approx(O.average_plaquette(U), abs=1e-12)


def test_fp32_iterations_track_fp64(lgf):
    """FP32 storage: after 10 iterations every link element is within FP32
    rounding growth (2e-5) of the FP64 oracle."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=0, link_scale=0.3)
    ref = O.iterate(U, 10, ALPHA)
    for dtype in ("f32", "f32_r12"):
        with lgf.GaugeFixer(dims, dtype) as gf:
            gf.load_links(U)
            gf.iterate(10)
            out = gf.store_links()
        assert np.max(np.abs(out - ref)) <= 2e-5, dtype


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_constant_links_stay_fixed(lgf):
    u = I.random_links((1, 1, 1, 1), 9, 1.3)[0, 0, 0, 0]
    dims = (4, 2, 6, 2)
    U = np.broadcast_to(u, I.lattice_shape(dims) + (4, 3, 3)).copy()
    with lgf.GaugeFixer(dims, "f64") as gf:
        gf.load_links(U)
        F, th = gf.functional()
        gf.iterate(3)
        out = gf.store_links()
        iters, conv = gf.fix(1e-20, 10)
    assert th < 1e-28
    assert np.max(np.abs(out - U)) < 1e-14
    assert conv and iters == 0


def test_zero_iterations_and_max_iter_zero(lgf):
    dims = (4, 4, 4, 4)
    U = I.synthetic_config(dims, seed=5, link_scale=0.5)
    with lgf.GaugeFixer(dims, "f64") as gf:
        gf.load_links(U)
        gf.iterate(0)
        assert np.array_equal(gf.store_links(), U)
        iters, conv = gf.fix(1e-12, 0)
        assert iters == 0 and not conv
        with pytest.raises(lgf.LgfError, match="NOT_CONVERGED"):
            gf.fix(1e-12, 0, raise_on_fail=True)


def test_nonfinite_links_are_reported(lgf):
    dims = (4, 4, 4, 4)
    U = I.synthetic_config(dims, seed=5, link_scale=0.5)
    U[1, 2, 3, 0, 2, 1, 1] = np.nan
    with lgf.GaugeFixer(dims, "f64") as gf:
        gf.load_links(U)
        with pytest.raises(lgf.LgfError, match="NONFINITE"):
            gf.functional()
        with pytest.raises(lgf.LgfError, match="NONFINITE"):
            gf.fix(1e-12, 10)


def test_bad_parameters_are_rejected(lgf):
    with lgf.GaugeFixer((4, 4, 4, 4), "f64") as gf:
        with pytest.raises(lgf.LgfError, match="ARG"):
            gf.set_param(0, 0.2)  # alpha > 1/8 is unstable
        with pytest.raises(lgf.LgfError, match="ARG"):
            gf.iterate(1)  # nothing loaded


def test_determinism(lgf):
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=7, link_scale=0.5)
    outs = []
    for _ in range(2):
        with lgf.GaugeFixer(dims, "f32") as gf:
            gf.load_links(U)
            gf.iterate(20)
            outs.append((gf.store_links(), gf.functional()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_device_tensor_load_and_torch_stream(lgf):
    import torch
    dims = (6, 4, 4, 10)
    U = I.synthetic_config(dims, seed=8, link_scale=0.5)
    ref = O.iterate(U, 5, ALPHA)
    s = torch.cuda.Stream()
    t = torch.from_numpy(U).to("cuda")
    torch.cuda.synchronize()
    with lgf.GaugeFixer(dims, "f64", stream=s) as gf:
        gf.load_links(t)
        gf.iterate(5)
        out = gf.store_links()
    assert np.max(np.abs(out - ref)) <= 1e-11


# ---------------------------------------------------------------------------
# full size, launch configuration of the benchmark (FP32 + FP64 tail, 32^4)
# ---------------------------------------------------------------------------

def test_full_size_32_4_fp32_tail(lgf):
    dims = (32, 32, 32, 32)
    U = I.synthetic_config(dims, seed=0, link_scale=0.5)
    rng = np.random.default_rng(0)
    shp = I.lattice_shape(dims)
    sites = tuple(rng.integers(0, n, 64) for n in shp)
    D_ref = O.gradient(U)
    plaq0 = O.average_plaquette(U)
    with lgf.GaugeFixer(dims, "f32") as gf:
        gf.load_links(U)
        pr = gf.probe()
        iters, conv = gf.fix(1e-15, 3000)
        F, th = gf.functional()
        out = gf.store_links()
    # FP32 gradient at sampled sites: |U| = 1 entries summed 8-fold in FP32
    np.testing.assert_allclose(pr["delta"][sites], _packed(D_ref)[sites], rtol=0, atol=5e-6)
    assert conv and th < 1e-15
    assert O.unitarity_defect(out) < 1e-12
    assert O.average_plaquette(out) == pytest.approx(plaq0, abs=1e-12)
    # Landau condition from the oracle's own gradient of the result
    assert O.functional(out)[1] < 1e-15
    assert F > O.functional(U)[0]
