"""CPU FP64 oracle for SU(3) Landau gauge fixing by steepest descent with
Fourier acceleration.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this module.  The product
library never calls it and shares no code with it: the GPU path packs the
traceless anti-Hermitian gradient into four complex fields and runs a
Stockham FFT; this oracle transforms each of the nine matrix entries on its
own with a naive, separable discrete Fourier transform, which is how the
paper's own GPU code treats the gradient (Sec. 2.2: every element of Delta is
transformed on its own, in place, in the structure-of-arrays layout).

The paper (Sec. 1) names the method -- steepest descent with Fourier
acceleration (Davies et al. 1988; Oliveira & Silva 2003) -- and Sec. 2.2 its
data flow (one thread per site, structure-of-arrays lattice, 4D FFT as 2D plus
2D).  It prints no formula of the iteration, so the iteration below is the
standard one of the cited method, in this notation:

* lattice ``L = (Lx, Ly, Lz, Lt)``, periodic, ``V = Lx Ly Lz Lt`` sites,
  ``N_c = 3`` colours, ``N_d = 4`` directions;
* gradient      A(x) = sum_mu [U_mu(x - mu) - U_mu(x)],
                Delta(x) = A - A^dagger - (1/3) Tr(A - A^dagger) * 1;
* functional    F = 1/(N_d N_c V) sum_{x,mu} Re Tr U_mu(x);
* convergence   theta = 1/(N_c V) sum_x Tr Delta Delta^dagger;
* acceleration  Delta~ = FFT^-1[ p2_max / p2(k) * FFT[Delta] ],
                p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu),
                p2_max = sum_mu max_k 4 sin^2(pi k / L_mu), and 0 at k = 0;
* gauge step    g(x) = reunitarised exp(alpha/2 * Delta~(x)); the default
                (exp_order = 1) takes the first-order expansion
                1 + alpha/2 Delta~ before reunitarising, exp_order = 0 the
                exact exponential;
* update        U_mu(x) <- g(x) U_mu(x) g(x + mu)^dagger.

Readings where the paper is silent (the same list is kept with the design
notes): no factor 1/2 in Delta; F normalised by N_d N_c V; the k = 0 mode is
dropped; the forward transform is e^{-i k x} and unnormalised, the inverse
e^{+i k x} / V; theta and F are those of the links *before* an update, and an
"iteration" is one applied update; reunitarisation is Gram-Schmidt on rows
one and two with row three = conj(row1 x row2).

Array layout: complex128 ``U[t, z, y, x, mu, i, j]`` (x fastest), direction
``mu = 0..3`` is x, y, z, t, so ``mu`` lives on array axis ``3 - mu``.

Every function is plain numpy in float64/complex128, written for checking by
eye, not for speed.
"""
from __future__ import annotations

import math

import numpy as np

N_C = 3
N_D = 4
AXIS = (3, 2, 1, 0)  # array axis of direction mu


def lattice_dims(U: np.ndarray):
    """(Lx, Ly, Lz, Lt) of a link or site array."""
    Lt, Lz, Ly, Lx = U.shape[:4]
    return (Lx, Ly, Lz, Lt)


def dagger(M: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(M, -1, -2))


def shift(field: np.ndarray, mu: int, step: int) -> np.ndarray:
    """field(x + step * mu) on the periodic lattice."""
    return np.roll(field, -step, axis=AXIS[mu])


# ---------------------------------------------------------------------------
# SU(3) projection (the "reunitarised" of the gauge step)
# ---------------------------------------------------------------------------

def reunitarize(M: np.ndarray) -> np.ndarray:
    """Project 3x3 matrices onto SU(3): Gram-Schmidt on rows 1 and 2, row 3 as
    the complex conjugate of their cross product (det = +1)."""
    r1 = M[..., 0, :]
    r2 = M[..., 1, :]
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    proj = np.sum(np.conj(r1) * r2, axis=-1)[..., None]
    r2 = r2 - proj * r1
    r2 = r2 / np.sqrt(np.sum(np.abs(r2) ** 2, axis=-1))[..., None]
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


# ---------------------------------------------------------------------------
# gradient, functional, convergence measure
# ---------------------------------------------------------------------------

def gradient(U: np.ndarray) -> np.ndarray:
    """Delta(x): traceless anti-Hermitian part (times 2) of
    A(x) = sum_mu [U_mu(x - mu) - U_mu(x)]."""
    A = np.zeros(U.shape[:4] + (3, 3), dtype=np.complex128)
    for mu in range(N_D):
        A += shift(U[..., mu, :, :], mu, -1) - U[..., mu, :, :]
    D = A - dagger(A)
    tr = np.trace(D, axis1=-2, axis2=-1) / 3.0
    return D - tr[..., None, None] * np.eye(3)


def functional(U: np.ndarray, Delta: np.ndarray | None = None):
    """(F, theta) of the links U."""
    V = int(np.prod(U.shape[:4]))
    if Delta is None:
        Delta = gradient(U)
    re_tr = np.real(np.trace(U, axis1=-2, axis2=-1))  # (..., mu)
    F = math.fsum(re_tr.ravel()) / (N_D * N_C * V)
    tr_dd = np.sum(np.abs(Delta) ** 2, axis=(-2, -1))  # Tr Delta Delta^dagger
    theta = math.fsum(tr_dd.ravel()) / (N_C * V)
    return F, theta


# ---------------------------------------------------------------------------
# Fourier acceleration
# ---------------------------------------------------------------------------

def dft_matrix(L: int, sign: int) -> np.ndarray:
    """W[k, j] = exp(sign * 2 pi i (j k mod L) / L)."""
    jk = np.outer(np.arange(L), np.arange(L)) % L
    ang = 2.0 * np.pi * jk / L
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dft4(field: np.ndarray, sign: int) -> np.ndarray:
    """Naive separable 4D DFT over the lattice axes of ``field`` (unnormalised).

    Each 1D transform is a direct O(L^2) sum, applied along t, z, y and x in
    turn; the trailing axes (matrix entries) are independent transforms.
    """
    out = field
    for ax in range(4):
        L = out.shape[ax]
        W = dft_matrix(L, sign)
        out = np.moveaxis(np.tensordot(W, out, axes=([1], [ax])), 0, ax)
    return out


def momentum_sq(dims) -> np.ndarray:
    """p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu), array of shape (Lt, Lz, Ly, Lx)."""
    Lx, Ly, Lz, Lt = dims
    per_axis = [4.0 * np.sin(np.pi * np.arange(n) / n) ** 2 for n in (Lt, Lz, Ly, Lx)]
    return (per_axis[0][:, None, None, None] + per_axis[1][None, :, None, None]
            + per_axis[2][None, None, :, None] + per_axis[3][None, None, None, :])


def p2_max(dims) -> float:
    return float(sum(np.max(4.0 * np.sin(np.pi * np.arange(n) / n) ** 2) for n in dims))


def acceleration_factor(dims, zero_mode: float = 0.0) -> np.ndarray:
    """K(k) = p2_max / p2(k), with K(0) = zero_mode (0 by default)."""
    p2 = momentum_sq(dims)
    K = np.empty_like(p2)
    nz = p2 > 0
    K[nz] = p2_max(dims) / p2[nz]
    K[~nz] = zero_mode
    return K


def accelerate(Delta: np.ndarray, accel: bool = True, zero_mode: float = 0.0) -> np.ndarray:
    """Delta~ = FFT^-1[K(k) FFT[Delta]] entry by entry (K = 1 if not accel)."""
    dims = lattice_dims(Delta)
    V = int(np.prod(Delta.shape[:4]))
    if not accel:
        return Delta.copy()
    Dk = dft4(Delta, -1)
    Dk = Dk * acceleration_factor(dims, zero_mode)[..., None, None]
    return dft4(Dk, +1) / V


# ---------------------------------------------------------------------------
# gauge step and update
# ---------------------------------------------------------------------------

def expm_antihermitian(X: np.ndarray) -> np.ndarray:
    """exp(X) for anti-Hermitian X through the eigen-decomposition of -iX."""
    H = -1j * X
    H = 0.5 * (H + dagger(H))
    w, v = np.linalg.eigh(H)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def gauge_step(Dt: np.ndarray, alpha: float, exp_order: int = 1) -> np.ndarray:
    """g(x) = reunitarised exp(alpha/2 Delta~(x))."""
    X = 0.5 * alpha * Dt
    if exp_order == 1:
        M = np.eye(3) + X
    elif exp_order == 0:
        M = expm_antihermitian(X)
    else:
        raise ValueError("exp_order must be 0 (exact) or 1 (first order)")
    return reunitarize(M)


def gauge_transform(U: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) <- g(x) U_mu(x) g(x + mu)^dagger, into a new array."""
    out = np.empty_like(U)
    gd = dagger(g)
    for mu in range(N_D):
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ shift(gd, mu, +1)
    return out


def step_parts(U: np.ndarray, alpha: float, exp_order: int = 1, accel: bool = True):
    """Every intermediate of one iteration, for step-by-step comparison."""
    Delta = gradient(U)
    F, theta = functional(U, Delta)
    Dt = accelerate(Delta, accel)
    g = gauge_step(Dt, alpha, exp_order)
    return {"Delta": Delta, "F": F, "theta": theta, "Delta_tilde": Dt, "g": g,
            "U_next": gauge_transform(U, g)}


def iterate(U: np.ndarray, n: int, alpha: float = 0.08, exp_order: int = 1,
            accel: bool = True, history: list | None = None) -> np.ndarray:
    """Apply exactly n updates.  If ``history`` is a list, (F, theta) of the
    links before each update is appended to it."""
    for _ in range(n):
        Delta = gradient(U)
        if history is not None:
            history.append(functional(U, Delta))
        g = gauge_step(accelerate(Delta, accel), alpha, exp_order)
        U = gauge_transform(U, g)
    return U


def fix(U: np.ndarray, theta_tol: float, max_iter: int, alpha: float = 0.08,
        exp_order: int = 1, accel: bool = True, track_gauge: bool = False):
    """Iterate until theta < theta_tol or max_iter updates have been applied.

    Returns a dict with the final links, the number of updates, F and theta of
    the final links, whether it converged, the (F, theta) history and, if
    ``track_gauge``, the accumulated transformation G with U_final =
    G(x) U_mu(x) G(x+mu)^dagger.
    """
    n = 0
    hist = []
    G = None
    if track_gauge:
        G = np.broadcast_to(np.eye(3, dtype=np.complex128), U.shape[:4] + (3, 3)).copy()
    while True:
        Delta = gradient(U)
        F, theta = functional(U, Delta)
        hist.append((F, theta))
        if theta < theta_tol or n == max_iter:
            break
        g = gauge_step(accelerate(Delta, accel), alpha, exp_order)
        U = gauge_transform(U, g)
        if track_gauge:
            G = g @ G
        n += 1
    return {"U": U, "iterations": n, "F": F, "theta": theta,
            "converged": theta < theta_tol, "history": hist, "G": G}


# ---------------------------------------------------------------------------
# gauge-invariant and structural checks used by the tests
# ---------------------------------------------------------------------------

def average_plaquette(U: np.ndarray) -> float:
    """(1/(6 N_c V)) sum_x sum_{mu<nu} Re Tr P_{mu nu}(x) (gauge invariant)."""
    V = int(np.prod(U.shape[:4]))
    tot = 0.0
    for mu in range(N_D):
        for nu in range(mu + 1, N_D):
            Umu = U[..., mu, :, :]
            Unu = U[..., nu, :, :]
            P = Umu @ shift(Unu, mu, +1) @ dagger(shift(Umu, nu, +1)) @ dagger(Unu)
            tot += math.fsum(np.real(np.trace(P, axis1=-2, axis2=-1)).ravel())
    return tot / (6 * N_C * V)


def unitarity_defect(M: np.ndarray) -> float:
    """max |M M^dagger - 1| and max |det M - 1| over all matrices."""
    eye = np.eye(3)
    d1 = np.max(np.abs(M @ dagger(M) - eye))
    d2 = np.max(np.abs(np.linalg.det(M) - 1.0))
    return float(max(d1, d2))


def pack_delta(Delta: np.ndarray) -> np.ndarray:
    """The 8 real degrees of freedom of a traceless anti-Hermitian matrix as 4
    complex numbers (D01, D02, D12, Im D00 + i Im D11): shape (..., 4).

    Used only to compare against the packed field the GPU stores; the oracle
    itself transforms all nine entries."""
    return np.stack([Delta[..., 0, 1], Delta[..., 0, 2], Delta[..., 1, 2],
                     np.imag(Delta[..., 0, 0]) + 1j * np.imag(Delta[..., 1, 1])], axis=-1)
