"""Pins of the warm-start oracle (oracle/warm_start_oracle.py): brute force,
finite differences and invariances, none of which re-types its formulas."""
import itertools

import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O
from oracle import warm_start_oracle as W


def test_su3_coefficients_round_trip():
    rng = np.random.default_rng(0)
    c = rng.standard_normal((5, 8))
    X = np.einsum("na,aij->nij", 0.5j * c, W.gell_mann())
    np.testing.assert_allclose(W.su3_coefficients(X), c, atol=1e-14)
    # the Hermitian and trace parts do not leak in
    H = rng.standard_normal((5, 3, 3)) + 1j * rng.standard_normal((5, 3, 3))
    H = H + O.dagger(H)
    np.testing.assert_allclose(W.su3_coefficients(X + H + 2j * np.eye(3)), c, atol=1e-13)


def _brute_conv(x, Wt, b):
    Lt, Lz, Ly, Lx, _ = x.shape
    y = np.zeros((Lt, Lz, Ly, Lx, Wt.shape[2]))
    for t, z, yy, xx in itertools.product(range(Lt), range(Lz), range(Ly), range(Lx)):
        acc = b.copy()
        for dt, dz, dy, dx in itertools.product((-1, 0, 1), repeat=4):
            tap = ((dt + 1) * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1))
            acc = acc + x[(t + dt) % Lt, (z + dz) % Lz, (yy + dy) % Ly, (xx + dx) % Lx] @ Wt[tap]
        y[t, z, yy, xx] = acc
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 2, 3, 4, 2))
    Wt = rng.standard_normal((81, 2, 3))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(W.conv(x, Wt, b), _brute_conv(x, Wt, b), atol=1e-12)


def test_conv_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 2, 3, 2))
    Wt = rng.standard_normal((81, 2, 3))
    b = rng.standard_normal(3)
    gy = rng.standard_normal(x.shape[:4] + (3,))
    gx, gW, gb = W.conv_backward(x, Wt, gy)
    f = lambda x_, W_, b_: float(np.sum(gy * W.conv(x_, W_, b_)))
    eps = 1e-6
    for idx in [(0, 0, 0, 0, 0), (1, 2, 1, 2, 1), (0, 1, 1, 0, 1)]:
        d = np.zeros_like(x); d[idx] = eps
        assert (f(x + d, Wt, b) - f(x - d, Wt, b)) / (2 * eps) == pytest.approx(gx[idx], rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0), (40, 1, 2), (80, 0, 1)]:
        d = np.zeros_like(Wt); d[idx] = eps
        assert (f(x, Wt + d, b) - f(x, Wt - d, b)) / (2 * eps) == pytest.approx(gW[idx], rel=1e-6, abs=1e-8)
    d = np.zeros_like(b); d[1] = eps
    assert (f(x, Wt, b + d) - f(x, Wt, b - d)) / (2 * eps) == pytest.approx(gb[1], rel=1e-6)


def test_network_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    shp = (2, 2, 3, 2)
    x0 = rng.standard_normal(shp + (W.N_FEAT,))
    params = [(0.05 * rng.standard_normal((81, W.N_FEAT, W.N_HID)), 0.1 * rng.standard_normal(W.N_HID)),
              (0.05 * rng.standard_normal((81, W.N_HID, W.N_HID)), 0.1 * rng.standard_normal(W.N_HID)),
              (0.05 * rng.standard_normal((81, W.N_HID, W.N_OUT)), 0.1 * rng.standard_normal(W.N_OUT))]
    R = rng.standard_normal(shp + (W.N_OUT,))
    c, acts = W.forward(x0, params)
    grads = W.backward(params, acts, R)
    f = lambda ps: float(np.sum(R * W.forward(x0, ps)[0]))
    eps = 1e-6
    for layer, idx in [(0, (3, 5, 7)), (1, (40, 10, 20)), (2, (80, 31, 5))]:
        Wp = [list(p) for p in params]
        Wm = [list(p) for p in params]
        Wp[layer][0] = params[layer][0].copy(); Wp[layer][0][idx] += eps
        Wm[layer][0] = params[layer][0].copy(); Wm[layer][0][idx] -= eps
        fd = (f(Wp) - f(Wm)) / (2 * eps)
        assert fd == pytest.approx(grads[layer][0][idx], rel=1e-5, abs=1e-9)


def test_training_signal_is_derivative_of_minus_F_at_identity():
    """At c = 0 the left-translation signal is the ordinary derivative."""
    dims = (3, 2, 4, 2)
    U = I.synthetic_config(dims, seed=4, link_scale=0.7)
    c = np.zeros(I.lattice_shape(dims) + (8,))
    L0, sig = W.loss_and_signal(U, c)
    assert L0 == pytest.approx(-O.functional(U)[0], rel=1e-14)
    eps = 1e-6
    for idx in [(0, 0, 0, 0, 0), (1, 3, 1, 2, 5), (0, 2, 1, 1, 7)]:
        d = np.zeros_like(c); d[idx] = eps
        fd = (W.loss_and_signal(U, c + d)[0] - W.loss_and_signal(U, c - d)[0]) / (2 * eps)
        assert fd == pytest.approx(sig[idx], rel=1e-6, abs=1e-12)


def test_features_plaquettes_are_gauge_invariant():
    dims = (2, 3, 2, 4)
    U = I.random_links(dims, 5, 0.6)
    g = I.random_gauge(dims, 6, 1.0)
    a, b = W.features(U), W.features(I.apply_gauge(U, g))
    np.testing.assert_allclose(a[..., 32:38], b[..., 32:38], atol=1e-13)
    assert np.all(W.features(np.broadcast_to(np.eye(3), U.shape).copy())[..., :32] == 0)
    np.testing.assert_allclose(W.features(np.broadcast_to(np.eye(3), U.shape).copy())[..., 32:38], 1.0)
