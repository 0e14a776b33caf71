"""The gauge transformation a fix has applied (lgf_store_gauge, LGF_TRACK_G)
on the GPU.

The fixed links must be G(x) U(x) G(x+mu)^dagger of the loaded links U, with
G in SU(3), as the oracle recomputes them from the stored G (its
gauge_transform is pinned by brute force in test_oracle.py).  For the FP64
path G is also compared with the oracle's own accumulated transformation
(O.fix(track_gauge=True)), which multiplies the same steps without
reunitarising in between: the two agree to rounding growth, 1e-10 like the
links after N iterations in test_gpu_parity.py."""
import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

pytestmark = pytest.mark.gpu

ALPHA = 0.08
LGF_TRACK_G = 9
LGF_TAIL_MODE = 7


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
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 10, 12)])
def test_fp64_tracked_gauge(lgf, dims, dtype):
    U = I.synthetic_config(dims, seed=1, link_scale=0.3)
    ref = O.fix(U, 1e-12, 2000, ALPHA, track_gauge=True)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.set_param(LGF_TRACK_G, 1)
        gf.load_links(U)
        it, conv = gf.fix(1e-12, 2000)
        G = gf.store_gauge()
        links = gf.store_links()
    assert conv and it == ref["iterations"]
    assert O.unitarity_defect(G) < 1e-13
    assert np.max(np.abs(O.gauge_transform(U, G) - links)) <= 1e-12
    assert np.max(np.abs(G - ref["G"])) <= 1e-10


def test_fp64_tracking_changes_nothing_else(lgf):
    """Tracking adds a kernel but leaves the links and the update count bit for bit."""
    dims = (8, 8, 8, 8)
    U = I.synthetic_config(dims, seed=4, link_scale=0.3)
    out = []
    for track in (0, 1):
        with lgf.GaugeFixer(dims, "f64") as gf:
            gf.set_param(LGF_TRACK_G, track)
            gf.load_links(U)
            out.append((gf.fix(1e-12, 2000), gf.store_links()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("dtype", ["f32", "f32_r12"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 10, 12)])
def test_mixed_precision_gauge(lgf, dims, dtype):
    """FP32 phase: G in FP32 (the links it forms agree to FP32 rounding of the
    loaded links); after the double-float tail: (1 + eta) G in FP64, which
    reproduces the stored FP64 links to 1e-12."""
    U = I.synthetic_config(dims, seed=2, link_scale=0.5)
    with lgf.GaugeFixer(dims, dtype) as gf:
        gf.load_links(U)
        gf.iterate(5)
        G5 = gf.store_gauge()
        l5 = gf.store_links()
        assert O.unitarity_defect(G5) < 1e-5
        assert np.max(np.abs(O.gauge_transform(U, G5) - l5)) <= 1e-5
        gf.load_links(U)
        _, conv = gf.fix(1e-15, 2000)
        assert conv and gf.fix_split()[1] > 0  # the double-float tail ran
        G = gf.store_gauge()
        links = gf.store_links()
        F, th = gf.functional()
    assert O.unitarity_defect(G) < 1e-13
    assert np.max(np.abs(O.gauge_transform(U, G) - links)) <= 1e-12
    F2, th2 = O.functional(O.gauge_transform(U, G))
    assert F2 == pytest.approx(F, rel=1e-12) and th2 < 1e-14


def test_untracked_gauge_is_refused(lgf):
    U = I.synthetic_config((4, 4, 4, 4), seed=0, link_scale=0.3)
    with lgf.GaugeFixer((4, 4, 4, 4), "f64") as gf:
        gf.load_links(U)
        with pytest.raises(lgf.LgfError):
            gf.store_gauge()
        gf.set_param(LGF_TRACK_G, 1)  # from the next load
        with pytest.raises(lgf.LgfError):
            gf.store_gauge()
        gf.load_links(U)
        gf.iterate(3)
        assert O.unitarity_defect(gf.store_gauge()) < 1e-13
    with lgf.GaugeFixer((4, 4, 4, 4), "f32") as gf:
        gf.set_param(LGF_TAIL_MODE, 1)  # the plain FP64 tail does not track G
        gf.load_links(U)
        gf.fix(1e-15, 2000)
        with pytest.raises(lgf.LgfError):
            gf.store_gauge()
