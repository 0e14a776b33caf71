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
import functools

import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu

ALPHA = 0.08

# FFT pipelines (LGF_FFT_PIPELINE): register planes where Lx = Ly and the
# (Lz, Lt) shape is instantiated; else per-axis register passes where every
# extent is in {4, 6, 8, 12, 16, 20, 24, 32}; else Stockham plane kernels.
STEP_DIMS = [
    (8, 8, 8, 8),      # C1 shape (register planes)
    (12, 12, 32, 8),   # register planes, z-t plane 32 x 8
    (32, 32, 8, 8),    # warp-tile x-y planes, one 32 x 32 tile per warp
    (16, 16, 32, 16),  # warp-tile x-y planes, two 16 x 16 tiles per warp
    (4, 4, 6, 6),      # warp-tile x-y planes, eight 4 x 4 tiles per warp
    (20, 20, 4, 4),    # warp-tile x-y planes, one 20 x 20 tile per warp, 12 lanes idle
    (24, 24, 6, 6),    # warp-tile x-y planes, one 24 x 24 tile per warp, 8 lanes idle
    (6, 6, 6, 6),      # warp-tile x-y planes, five 6 x 6 tiles per warp, 2 lanes idle
    (48, 48, 4, 4),    # two-warp x-y tiles (48 lines), fused inverse x-y + G update
    (6, 12, 4, 20),    # axis passes, radices 2, 3, 4, 5; V = 5760
    (20, 8, 24, 6),    # axis passes, V = 23040
    (4, 6, 10, 12),    # plane kernels (10); V = 2880, ragged last block
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


@functools.lru_cache(maxsize=None)
def _oracle_fix(dims, seed, link_scale, tol):
    U = I.synthetic_config(dims, seed=seed, link_scale=link_scale)
    return U, O.fix(U, tol, 2000, ALPHA)


@pytest.mark.parametrize("planes", [0, 1, 2, 3])
@pytest.mark.parametrize("dtype", ["f64", "f64_r12"])
@pytest.mark.parametrize("dims", STEP_DIMS)
def test_one_step_matches_oracle(lgf, dims, dtype, planes):
    U = I.synthetic_config(dims, seed=3, link_scale=0.5)
    ref = O.step_parts(U, ALPHA)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.set_param(5, planes)  # LGF_FFT_PIPELINE: auto, Stockham, axis passes, register planes
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


@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
@pytest.mark.parametrize("dims", STEP_DIMS)
def test_fp32_step_matches_oracle(lgf, dims, dtype):
    """One step of the FP32 engine (gauge representation, 18 or 12 reals)
    against the FP64 oracle on the same shapes.  Tolerances: rounding the
    input links to FP32 alone moves the oracle's Delta by ~3e-7 (|Delta| up
    to ~14), its Delta~ by ~2e-8 of max |Delta~|, g by ~3e-8 and the next
    links by ~6e-8; the FP32 products (27 MACs per product, ten products per
    site) and the FP32 FFT (~eps log2 V) add about an order of magnitude.  The
    bounds on Delta and Delta~ sit 10-50 times above that; F and theta carry
    FP64 sums above the warp.  g = reunit(1 + (alpha/2) Delta~) moves by at
    most alpha/2 times the error of Delta~ plus its own FP32 rounding, and the
    next links g U g'^dag by twice that (the acceleration factor reaches
    p2_max / (4 sin^2(pi/64)) ~ 1700 on 64-long lines, so there Delta~ and g
    carry the largest absolute errors)."""
    U = I.synthetic_config(dims, seed=3, link_scale=0.5)
    ref = O.step_parts(U, ALPHA)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        out = gf.probe()
        F, th = gf.functional()
        gf.iterate(1)
        U1 = gf.store_links()
    d_ref, dt_ref = _packed(ref["Delta"]), _packed(ref["Delta_tilde"])
    tol_dt = 4e-6 * np.max(np.abs(dt_ref))
    tol_g = ALPHA / 2 * tol_dt + 1e-6
    assert np.max(np.abs(out["delta"] - d_ref)) <= 2e-6 * np.max(np.abs(d_ref))
    assert np.max(np.abs(out["delta_tilde"] - dt_ref)) <= tol_dt
    np.testing.assert_allclose(out["g"], ref["g"], rtol=0, atol=tol_g)
    assert F == pytest.approx(ref["F"], rel=2e-6)
    assert th == pytest.approx(ref["theta"], rel=2e-5)
    np.testing.assert_allclose(U1, ref["U_next"], rtol=0, atol=2 * tol_g + 1e-6)


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


@pytest.mark.parametrize("link_update", [0, 1])
@pytest.mark.parametrize("reunit_fp64", [0, 1])
@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 10, 12), (16, 12, 8, 48), (8, 8, 32, 16)])
def test_mixed_precision_fix_matches_fp64_functional(lgf, dims, dtype, reunit_fp64, link_update):
    U, ref = _oracle_fix(dims, 2, 0.5, 1e-15)
    assert ref["converged"]
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.set_param(4, reunit_fp64)  # LGF_REUNIT_FP64
        gf.set_param(6, link_update)  # LGF_LINK_UPDATE: 0 gauge representation, 1 links in place
        gf.load_links(U)
        iters, conv = gf.fix(1e-15, 2000)
        F, th = gf.functional()
        out = gf.store_links()
    assert conv and th < 1e-15
    assert F == pytest.approx(ref["F"], rel=1e-12)
    assert O.unitarity_defect(out) < 1e-12
    assert O.average_plaquette(out) == pytest.approx(O.average_plaquette(U), abs=1e-12)


@pytest.mark.parametrize("link_update", [0, 1])
@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
def test_fp32_iterations_track_fp64(lgf, dtype, link_update):
    """FP32 storage: after 10 iterations every link element is within FP32
    rounding growth (2e-5) of the FP64 oracle, in both update modes; one step
    matches the oracle's intermediates to FP32 rounding.  The accelerated
    gradient goes through a forward and an inverse FFT over V = 4096 points
    in FP32: its error is a few eps * log2(V) ~ 4e-6 of its largest entry
    (the acceleration makes |Delta~| reach ~20 here)."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=0, link_scale=0.3)
    ref = O.iterate(U, 10, ALPHA)
    parts = O.step_parts(U, ALPHA)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.set_param(6, link_update)
        gf.load_links(U)
        pr = gf.probe()
        F, th = gf.functional()
        gf.iterate(10)
        out = gf.store_links()
    np.testing.assert_allclose(pr["delta"], _packed(parts["Delta"]), rtol=0, atol=5e-6)
    dt_ref = _packed(parts["Delta_tilde"])
    np.testing.assert_allclose(pr["delta_tilde"], dt_ref, rtol=0, atol=4e-6 * np.max(np.abs(dt_ref)))
    np.testing.assert_allclose(pr["g"], parts["g"], rtol=0, atol=1e-6)
    assert F == pytest.approx(parts["F"], rel=1e-6)
    assert th == pytest.approx(parts["theta"], rel=1e-5)
    assert np.max(np.abs(out - ref)) <= 2e-5


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


@pytest.mark.parametrize("link_update", [0, 1])
def test_determinism(lgf, link_update):
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=7, link_scale=0.5)
    outs = []
    for _ in range(2):
        with lgf.GaugeFixer(dims, "f32") as gf:
            gf.set_param(6, link_update)
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
    # the oracle's own fix of this input (stored by tests/golden/make_fullsize_fix.py)
    from tests.test_gpu_fullsize import check_against_oracle_fix
    check_against_oracle_fix("32^4", dims, F, iters)


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (12, 12, 32, 8)])
def test_both_fp64_tails_reach_the_oracle_functional(lgf, dims):
    """LGF_TAIL_MODE 0 (defect-correction tail on double-float links), 2 (the
    same tail on FP64 links) and 1 (plain FP64 iteration) all end at the
    oracle's FP64 functional to 1e-12 relative, with theta < 1e-15."""
    U, ref = _oracle_fix(dims, 2, 0.5, 1e-15)
    res = {}
    for mode in (0, 2, 1):
        with lgf.GaugeFixer(dims, "f32") as gf:
            gf.set_param(7, mode)  # LGF_TAIL_MODE
            gf.load_links(U)
            iters, conv = gf.fix(1e-15, 2000)
            F, th = gf.functional()
            res[mode] = (iters, gf.fix_split(), F, gf.store_links())
        assert conv and th < 1e-15
        assert F == pytest.approx(ref["F"], rel=1e-12)
    assert res[0][1][0] == res[1][1][0] == res[2][1][0]  # the same FP32 phase
    if res[0][1] == res[2][1]:
        # the double-float and FP64 forms of the defect tail take the same
        # steps: their FP32 corrections differ by at most an FP32 rounding of
        # a correction (|eps| 2^-24 < 1e-11), their link storage by 2^-47
        assert np.max(np.abs(res[0][3] - res[2][3])) < 1e-10

@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (12, 12, 32, 8)])
def test_double_float_tail_start_matches_the_fp64_one(lgf, dims, dtype):
    """The tail start alone: a fix capped at the FP32 phase's own length runs
    that phase, rebuilds the links from the loaded input as G U G'^dag and
    stops.  In tail mode 0 G is reunitarised and the product formed in
    double-float (48-bit significands), in mode 2 in FP64: the links agree to
    a few 2^-47 per entry.  Mode 2 is unitary to FP64 rounding; the
    double-float links carry a representation error of up to 2^-48 per real,
    and det U sums six triple products of them, so their defect bound is
    6 x 3 x 2 x 2^-48 ~ 1.3e-13."""
    U = I.synthetic_config(dims, seed=3, link_scale=0.5)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        gf.fix(1e-15, 2000)
        n32 = gf.fix_split()[0]
    out = {}
    for mode in (0, 2):
        with lgf.GaugeFixer(dims, dtype) as gf:
            gf.set_param(7, mode)  # LGF_TAIL_MODE
            gf.load_links(U)
            it, conv = gf.fix(1e-15, n32)
            assert it == n32 and not conv
            out[mode] = gf.store_links()
    assert np.max(np.abs(out[0] - out[2])) < 5e-14
    assert O.unitarity_defect(out[0]) < 1.3e-13
    assert O.unitarity_defect(out[2]) < 5e-14


@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
def test_tail_links_read_the_same_before_and_after_conversion(lgf, dtype):
    """After the double-float tail the handle holds its links as the tail
    start's double-float links and the tail's gauge transformation 1 + eta.
    lgf_store_links and lgf_functional form them on the fly; lgf_probe first
    applies eta and converts them to FP64 planes.  Both readings agree to
    FP64 rounding, and a later fix continues from either."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=4, link_scale=0.5)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        it, conv = gf.fix(1e-15, 2000)
        assert conv and gf.fix_split()[1] > 0
        F1, th1 = gf.functional()
        out1 = gf.store_links()
        gf.probe()
        F2, th2 = gf.functional()
        out2 = gf.store_links()
        it2, conv2 = gf.fix(1e-15, 2000)
    assert np.max(np.abs(out1 - out2)) < 1e-14
    assert F2 == pytest.approx(F1, rel=1e-14)
    assert th1 < 1e-15 and th2 < 1e-15 and abs(th1 - th2) < 1e-18
    assert conv2 and it2 == 0
    assert O.functional(out1)[1] < 1e-15


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_device_loop_and_host_loop_stop_at_the_same_update(lgf, mode):
    """lgf_fix runs each phase as a device-side graph loop, or (under
    lgf_profile) as host-queued iterations; both apply the same on-device stop
    rule, so they stop at the same update with bit-identical links."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=5, link_scale=0.5)
    out = []
    for profiled in (False, True):
        with lgf.GaugeFixer(dims, "f32") as gf:
            gf.set_param(7, mode)  # LGF_TAIL_MODE
            gf.load_links(U)
            gf.profile(profiled)
            it, conv = gf.fix(1e-15, 2000)
            out.append((it, conv, gf.fix_split(), gf.store_links(), gf.history()))
    assert out[0][:3] == out[1][:3]
    assert np.array_equal(out[0][3], out[1][3])
    assert np.array_equal(out[0][4], out[1][4])


def test_fp32_stall_rule_hands_over_the_same_way_in_both_loops(lgf):
    """With a hand-over threshold FP32 cannot reach, the FP32 phase ends by the
    stall rule (theta below 1e-6 not halving within 8 updates), applied on
    the device after every update; both loops hand over at the same update and
    the tail still reaches the oracle's functional."""
    dims = (8, 8, 8, 8)
    U, ref = _oracle_fix(dims, 2, 0.5, 1e-15)
    out = []
    for profiled in (False, True):
        with lgf.GaugeFixer(dims, "f32") as gf:
            gf.set_param(2, 1e-16)  # LGF_TAIL_THETA below the FP32 floor
            gf.load_links(U)
            gf.profile(profiled)
            it, conv = gf.fix(1e-15, 2000)
            F, th = gf.functional()
            out.append((it, gf.fix_split(), gf.store_links()))
            assert conv and th < 1e-15
            assert F == pytest.approx(ref["F"], rel=1e-12)
    assert out[0][:2] == out[1][:2]
    n32 = out[0][1][0]
    assert 0 < n32 < 2000  # the FP32 phase stopped by the stall rule, not the budget
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("dtype", ["f64", "f32", "f32_r12"])
def test_pinned_host_buffers_match_pageable_ones(lgf, dtype):
    """Loads from and stores to pinned host memory go straight through the
    layout kernels (the device reads and writes the host array); pageable
    arrays go through a staging copy.  Both give bit-identical links, after
    iterations (FP32: links formed from G) and after a fix (FP64 links)."""
    import torch
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=7, link_scale=0.5)
    pin_in = torch.empty(U.shape + (2,), dtype=torch.float64, pin_memory=True)
    pin_out = torch.empty(U.shape + (2,), dtype=torch.float64, pin_memory=True)
    assert pin_in.is_pinned() and pin_out.is_pinned()
    hin = pin_in.numpy().view(np.complex128).reshape(U.shape)
    hout = pin_out.numpy().view(np.complex128).reshape(U.shape)
    hin[...] = U
    with lgf.GaugeFixer(dims, dtype) as a, lgf.GaugeFixer(dims, dtype) as b:
        a.load_links(U)
        b.load_links(hin)
        for step in ("iterate", "fix"):
            if step == "iterate":
                a.iterate(5)
                b.iterate(5)
            else:
                a.fix(1e-12, 2000)
                b.fix(1e-12, 2000)
            ref = a.store_links()
            hout[...] = 0
            b.store_links(hout)
            assert np.array_equal(ref, hout), step
