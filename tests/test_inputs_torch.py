"""The torch (GPU-capable) generator reproduces the numpy recipe.  Runs on the
CPU here (torch on the host), on the GPU in the gpu-marked test."""
import numpy as np
import pytest

import lgf_inputs as I

torch = pytest.importorskip("torch")
from lgf_inputs import torch_gen as TG  # noqa: E402


def test_normal_deviates_match_numpy_bits_of_counters():
    a = I.normal_deviates(5, 1, 300, 4)
    b = TG.normal_deviates(5, 1, 300, 4, "cpu").numpy()
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims", [(2, 3, 4, 2), (4, 4, 4, 6)])
def test_config_matches_numpy(dims):
    a = I.synthetic_config(dims, seed=3, link_scale=0.6, gauge_scale=1.0)
    b = TG.synthetic_config(dims, seed=3, link_scale=0.6, gauge_scale=1.0, device="cpu").numpy()
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-13)


@pytest.mark.gpu
def test_config_matches_numpy_on_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dims = (6, 4, 8, 4)
    a = I.synthetic_config(dims, seed=9, link_scale=0.5)
    b = TG.synthetic_config(dims, seed=9, link_scale=0.5, device="cuda").cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-13)
