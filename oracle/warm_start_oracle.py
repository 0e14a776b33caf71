"""CPU FP64 oracle for the learned warm start of Landau gauge fixing.

TEST INFRASTRUCTURE (same rules as lgf_oracle: only tests/, smoke() and the
CPU baseline of bench.py use it).  It defines, in plain numpy, what the GPU
warm-start kernels compute:

* features(U): per site, the 8 su(3) coefficients of the traceless
  anti-Hermitian part of each of the 4 links (32 channels), the real parts of
  the 6 plaquette traces divided by 3 (gauge invariant), zero-padded to 48;
* a 4D convolution layer on the periodic lattice with 3^4 taps,
  y[s, o] = b[o] + sum_{tap, i} W[tap, i, o] x[s + off(tap), i], tap =
  ((dt*3 + dz)*3 + dy)*3 + dx with offsets d - 1 in {-1, 0, 1}; ReLU after
  layers 1 and 2; its gradients with respect to x, W and b;
* the warm start g0(x) = exp(X(x)), X = sum_a c_a(x) i lambda_a / 2, from the
  network's 8 outputs c_a;
* the training signal: F(U^{g0}) is the method's own functional.  Moving
  g0(x) to exp(eps Y) g0(x) changes F by eps <Y, Delta'(x)> / (2 N_d N_c V),
  with Delta' the gradient of the transformed links (the same identity the
  oracle tests pin by finite differences).  The loss is L = -F(U^{g0}) and the
  signal fed back into the network is dL/dc_a(x) taken along left
  translations, -<i lambda_a/2, Delta'(x)> / (24 V) (exact for small X).

The paper (Sec. 1) uses the plain method only; the warm start is the learned
extension this build adds (its readings are listed with the design notes).
"""
from __future__ import annotations

import numpy as np

from . import lgf_oracle as O


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices (written out here, not imported from the
    input generator, so the oracle stands alone)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


N_FEAT = 48
N_HID = 32
N_OUT = 8


def su3_coefficients(M: np.ndarray) -> np.ndarray:
    """c_a with sum_a c_a i lambda_a/2 = traceless anti-Hermitian part of M,
    (M - M^dag)/2 - trace; c_a = -i Tr(lambda_a A) for that part A."""
    A = 0.5 * (M - O.dagger(M))
    A = A - (np.trace(A, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
    lam = gell_mann()
    return np.real(-1j * np.einsum("aij,...ji->...a", lam, A))


def features(U: np.ndarray) -> np.ndarray:
    """(Lt, Lz, Ly, Lx, 48) float64 input of the network."""
    shp = U.shape[:4]
    out = np.zeros(shp + (N_FEAT,))
    for mu in range(4):
        out[..., 8 * mu:8 * mu + 8] = su3_coefficients(U[..., mu, :, :])
    k = 32
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Umu, Unu = U[..., mu, :, :], U[..., nu, :, :]
            P = Umu @ O.shift(Unu, mu, +1) @ O.dagger(O.shift(Umu, nu, +1)) @ O.dagger(Unu)
            out[..., k] = np.real(np.trace(P, axis1=-2, axis2=-1)) / 3.0
            k += 1
    return out


def tap_offsets():
    """(dx, dy, dz, dt) in {-1, 0, 1} for tap = ((dt*3 + dz)*3 + dy)*3 + dx."""
    offs = []
    for tap in range(81):
        dx, dy, dz, dt = tap % 3 - 1, (tap // 3) % 3 - 1, (tap // 9) % 3 - 1, tap // 27 - 1
        offs.append((dx, dy, dz, dt))
    return offs


def _shifted(x: np.ndarray, off) -> np.ndarray:
    """x[s + off] on the periodic lattice, x of shape (Lt, Lz, Ly, Lx, C)."""
    dx, dy, dz, dt = off
    return np.roll(x, shift=(-dt, -dz, -dy, -dx), axis=(0, 1, 2, 3))


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[s, o] = b[o] + sum_tap sum_i W[tap, i, o] x[s + off(tap), i]."""
    y = np.broadcast_to(b, x.shape[:4] + (W.shape[2],)).copy()
    for tap, off in enumerate(tap_offsets()):
        y += _shifted(x, off) @ W[tap]
    return y


def conv_backward(x: np.ndarray, W: np.ndarray, gy: np.ndarray):
    """Gradients (gx, gW, gb) of sum(gy * conv(x, W, b))."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for tap, off in enumerate(tap_offsets()):
        xs = _shifted(x, off)
        gW[tap] = xs.reshape(-1, xs.shape[-1]).T @ gy.reshape(-1, gy.shape[-1])
        # x[s + off] feeds y[s]: shift the contribution back by -off
        back = tuple(-o for o in off)
        gx += _shifted(gy @ W[tap].T, back)
    gb = gy.sum(axis=(0, 1, 2, 3))
    return gx, gW, gb


def forward(x0: np.ndarray, params):
    """Three layers, ReLU after the first two.  Returns the 8 outputs and the
    activations (for backward)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    z1 = conv(x0, W1, b1)
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, W2, b2)
    a2 = np.maximum(z2, 0.0)
    c = conv(a2, W3, b3)
    return c, (x0, z1, a1, z2, a2)


def backward(params, acts, gc):
    """Parameter gradients for upstream gradient gc = dL/dc."""
    (W1, b1), (W2, b2), (W3, b3) = params
    x0, z1, a1, z2, a2 = acts
    ga2, gW3, gb3 = conv_backward(a2, W3, gc)
    gz2 = ga2 * (z2 > 0)
    ga1, gW2, gb2 = conv_backward(a1, W2, gz2)
    gz1 = ga1 * (z1 > 0)
    _, gW1, gb1 = conv_backward(x0, W1, gz1)
    return [(gW1, gb1), (gW2, gb2), (gW3, gb3)]


def warm_gauge(c: np.ndarray) -> np.ndarray:
    """g0 = exp(sum_a c_a i lambda_a / 2) per site."""
    lam = gell_mann()
    X = np.einsum("...a,aij->...ij", 0.5j * c, lam)
    return O.expm_antihermitian(X)


def loss_and_signal(U: np.ndarray, c: np.ndarray):
    """L = -F(U^{g0}) and dL/dc along left translations,
    -<i lambda_a/2, Delta'> / (2 N_d N_c V) with <A, B> = Re Tr A^dag B."""
    g0 = warm_gauge(c)
    Up = O.gauge_transform(U, g0)
    D = O.gradient(Up)
    F, _ = O.functional(Up, D)
    V = int(np.prod(U.shape[:4]))
    lam = gell_mann()
    # <i lambda_a/2, D> = Re Tr[(i lambda_a/2)^dag D] = Re Tr[-i lambda_a D / 2]
    proj = np.real(np.einsum("aij,...ji->...a", -0.5j * lam, D))
    return -F, -proj / (2 * 4 * 3 * V)
