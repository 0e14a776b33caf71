"""The rule the library's exact gauge step uses for exp(X) (LGF_EXP_ORDER = 0,
expm_taylor in csrc/lgf_common.cuh), restated in numpy and checked against
scipy's expm: halve X until its squared Frobenius norm is at most 1/4, sum
the Taylor series by Horner's rule to degree 16 (FP64) or 9 (FP32), square
back.  This pins the choice of degree and scaling for the traceless
anti-Hermitian steps alpha/2 Delta~ the method produces (|X| up to ~2 on
small lattices, where the acceleration factor is large); the GPU kernels
themselves are held to the oracle in test_gpu_exp_order.py."""
import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")


def _expm_taylor(X: np.ndarray, dtype, degree: int) -> np.ndarray:
    X = X.astype(dtype)
    real = np.float64 if dtype == np.complex128 else np.float32
    n2 = real(np.sum(np.abs(X) ** 2))
    q, sc = 0, real(1)
    while n2 > real(0.25) and q < 30:
        n2 *= real(0.25)
        sc *= real(0.5)
        q += 1
    Y = X * sc
    eye = np.eye(3, dtype=dtype)
    E = eye.copy()
    for k in range(degree, 0, -1):
        E = eye + (Y @ E) * real(1.0 / k)
    for _ in range(q):
        E = E @ E
    return E


def _traceless_antihermitian(rng, norm):
    A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    X = A - A.conj().T
    X -= np.trace(X) / 3 * np.eye(3)
    return X * (norm / np.linalg.norm(X))


@pytest.mark.parametrize("norm", [1e-8, 1e-3, 0.1, 0.5, 1.0, 2.0, 3.0])
def test_taylor_rule_reaches_fp64_accuracy(norm):
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(50):
        X = _traceless_antihermitian(rng, norm)
        worst = max(worst, np.max(np.abs(_expm_taylor(X, np.complex128, 16) - scipy_linalg.expm(X))))
    assert worst < 2e-15


@pytest.mark.parametrize("norm", [1e-6, 0.1, 0.5, 1.0, 2.0])
def test_taylor_rule_reaches_fp32_accuracy(norm):
    """Degree 9 in FP32 arithmetic: within a few FP32 ulp of the exact
    exponential (its truncation error, 0.5^10 / 10! ~ 3e-10, is far below)."""
    rng = np.random.default_rng(8)
    worst = 0.0
    for _ in range(50):
        X = _traceless_antihermitian(rng, norm)
        worst = max(worst, np.max(np.abs(_expm_taylor(X, np.complex64, 9) - scipy_linalg.expm(X))))
    assert worst < 2e-6


def test_lower_degree_would_not_do():
    """The degree matters: at |X|_F = 1/2 after scaling, degree 8 leaves a
    truncation error above FP64 rounding, so the FP64 degree cannot be cut
    that far."""
    rng = np.random.default_rng(9)
    X = _traceless_antihermitian(rng, 0.5)
    ref = scipy_linalg.expm(X)
    assert np.max(np.abs(_expm_taylor(X, np.complex128, 8) - ref)) > 1e-12
    assert np.max(np.abs(_expm_taylor(X, np.complex128, 16) - ref)) < 2e-15
