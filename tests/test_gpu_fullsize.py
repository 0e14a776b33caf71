"""GPU parity at the full sizes of the paper-shaped workloads, in the launch
configuration the benchmark times.

The oracle needs minutes to fix one of these lattices, so its own fix of
each input is stored in ``tests/golden/fullsize_fix.json`` by the committed
script ``tests/golden/make_fullsize_fix.py``, which calls only the oracle and
the input generator.  Each test checks:
- the final functional F against the oracle's fix of the same input, to
  1e-12 relative (the acceptance bar of the mixed-precision path), and the
  number of updates against the oracle's;
- the FP32 gradient of the loaded links at sampled sites, against the
  oracle's FP64 gradient;
- properties of the fixed links: theta < 1e-15 recomputed by the oracle from
  the GPU's output (the Landau condition itself), the average plaquette of
  the input (a gauge-invariant quantity, so the output lies on the input's
  gauge orbit), unitarity, and a functional above the input's.
A batched fix must also reproduce a member's individual fix bit for bit.

The inputs here come from the GPU generator (``lgf_inputs.torch_gen``),
which matches the numpy generator the oracle ran on to about 1e-13 per
entry; that moves the final F by about as much, well inside 1e-12.
"""
import json
import os

import numpy as np
import pytest

from oracle import lgf_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_fix.json")


def golden_fix(case):
    """The oracle's fix of a full-size case: dims, seed, iterations, F, theta."""
    with open(GOLDEN) as f:
        rec = json.load(f)["cases"][case]
    assert rec["converged"] and rec["theta"] < 1e-15
    return rec


def check_against_oracle_fix(case, dims, F_gpu, iters_gpu):
    """Final F within 1e-12 relative of the oracle's own fix; the update
    count within 2 of the oracle's (the mixed path's FP32 phase and tail
    are a different arithmetic of the same iteration, so the count may
    differ where theta crosses 1e-15 between two updates)."""
    rec = golden_fix(case)
    assert tuple(rec["dims"]) == tuple(dims)
    assert F_gpu == pytest.approx(rec["F"], rel=1e-12), (F_gpu, rec["F"])
    assert abs(iters_gpu - rec["iterations"]) <= 2, (iters_gpu, rec["iterations"])


pytestmark = pytest.mark.gpu

# the batched workload: 64 members, 16 of each shape, seeds 0..63
BATCH_SHAPES = [(16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 8), (20, 20, 20, 20)]


@pytest.fixture(scope="module")
def lgf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1208_1186_gb300 as P
    from paper_1208_1186_gb300.build import build
    build()
    return P


def _device_config(dims, seed, link_scale):
    from lgf_inputs import torch_gen
    return torch_gen.synthetic_config(dims, seed=seed, link_scale=link_scale, gauge_scale=1.0, device="cuda")


def _check_fixed(out, U, F_gpu):
    """The fixed links out of input U: the Landau condition by the oracle's
    own gradient, the gauge orbit by the plaquette, unitarity, and F up."""
    F_out, th_out = O.functional(out)
    assert th_out < 1e-15
    assert O.unitarity_defect(out) < 1e-12
    assert O.average_plaquette(out) == pytest.approx(O.average_plaquette(U), abs=1e-12)
    assert F_gpu == pytest.approx(F_out, rel=1e-12)
    assert F_out > O.functional(U)[0]


@pytest.mark.parametrize("lt", [8, 12])
def test_full_size_48_cubed_r12(lgf, lt):
    """48^3 x 8 and 48^3 x 12 with 12-real FP32 links and link scale 0.6:
    two-warp x-y tiles (48-point lines), the fused inverse x-y + G update,
    and the double-float tail."""
    dims = (48, 48, 48, lt)
    Ud = _device_config(dims, 0, 0.6)
    U = Ud.cpu().numpy()
    rng = np.random.default_rng(1)
    sites = tuple(rng.integers(0, n, 64) for n in U.shape[:4])
    with lgf.GaugeFixer(dims, "f32_r12") as gf:
        gf.load_links(Ud)
        pr = gf.probe()
        iters, conv = gf.fix(1e-15, 3000)
        F, th = gf.functional()
        out = gf.store_links()
    # FP32 gradient (row 3 rebuilt in FP32) at sampled sites
    D_ref = O.pack_delta(O.gradient(U))
    np.testing.assert_allclose(pr["delta"][sites], D_ref[sites], rtol=0, atol=5e-6)
    assert conv and th < 1e-15
    _check_fixed(out, U, F)
    check_against_oracle_fix(f"48^3x{lt}", dims, F, iters)


def test_full_batch_of_64_mixed_shapes(lgf):
    """The whole batched workload fixed together, lanes autotuned: every
    member converges; one member of each shape is checked against the oracle
    and its individual fix."""
    n = 64
    shapes = [BATCH_SHAPES[i % len(BATCH_SHAPES)] for i in range(n)]
    inputs = [_device_config(shapes[i], i, 0.5) for i in range(n)]
    fixers = [lgf.GaugeFixer(shapes[i], "f32") for i in range(n)]
    try:
        for f, u in zip(fixers, inputs):
            f.load_links(u)
        with lgf.GaugeBatch(fixers) as b:
            b.autotune(reps=2)
            for f, u in zip(fixers, inputs):  # the autotuner iterated the members
                f.load_links(u)
            its, convs = b.fix(1e-15, 5000)
        assert all(convs)
        for f in fixers:
            assert f.functional()[1] < 1e-15
        for k in range(len(BATCH_SHAPES)):
            out = fixers[k].store_links()
            U = inputs[k].cpu().numpy()
            _check_fixed(out, U, fixers[k].functional()[0])
            Lx, _, _, Lt = shapes[k]
            name = f"{Lx}^4" if Lt == Lx else f"{Lx}^3x{Lt}"
            check_against_oracle_fix(f"batch member {k} {name}", shapes[k], fixers[k].functional()[0], its[k])
            with lgf.GaugeFixer(shapes[k], "f32") as gf:
                gf.load_links(inputs[k])
                it, conv = gf.fix(1e-15, 5000)
                assert it == its[k] and conv
                assert np.array_equal(gf.store_links(), out)
    finally:
        for f in fixers:
            f.close()
