"""Seeded synthetic SU(3) gauge configurations.

This module is the only code shared by the CPU oracle (``oracle/``) and the
GPU path (``paper_1208_1186_gb300``).  It produces *inputs* and holds none of
the gauge-fixing method's arithmetic: no gradient, no Fourier transform, no
reunitarisation and no functional.

Recipe (the paper fixes no generator; it gauge-fixes thermalised ensembles
that are not available here, so these configurations stand in for them):

* Random numbers: a counter-based generator.  Every normal deviate r is a pure
  function of ``(seed, stream, site, mu, a)``: the key is hashed with
  SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) and two hashes give one Box-Muller deviate.  The
  result is the same on every machine and every numpy version.
* Links: ``U_mu(x) = exp(i * scale * sum_a r_a lambda_a / 2)`` with the eight
  Gell-Mann matrices ``lambda_a`` (Tr lambda_a lambda_b = 2 delta_ab).  The
  exponential of the Hermitian traceless matrix is taken through its
  eigen-decomposition, so the result is unitary and has unit determinant to
  rounding; projecting it back onto SU(3) would change nothing.
* A random gauge transformation ``g(x)`` drawn the same way (stream 1, mu = 0)
  is then applied: ``U_mu(x) <- g(x) U_mu(x) g(x + mu)^dagger``.  This puts the
  configuration far from Landau gauge without changing any gauge-invariant
  quantity.

Layout: complex128 arrays of shape ``(Lt, Lz, Ly, Lx, 4, 3, 3)``; the site
index is ``s = x + Lx*(y + Ly*(z + Lz*t))`` (x fastest) and direction
``mu = 0, 1, 2, 3`` is x, y, z, t.  This is the host array-of-structures form
that ``lgf_load_links`` accepts.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "normal_deviates",
    "su3_from_coefficients",
    "random_gauge",
    "random_links",
    "apply_gauge",
    "synthetic_config",
    "lattice_shape",
]

_U64 = np.uint64
_GOLDEN = _U64(0x9E3779B97F4A7C15)
_MIX1 = _U64(0xBF58476D1CE4E5B9)
_MIX2 = _U64(0x94D049BB133111EB)


def lattice_shape(L):
    """Array shape ``(Lt, Lz, Ly, Lx)`` for ``L = (Lx, Ly, Lz, Lt)``."""
    Lx, Ly, Lz, Lt = (int(v) for v in L)
    return (Lt, Lz, Ly, Lx)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
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


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of ``z + golden`` (wrapping uint64 arithmetic)."""
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> _U64(30))) * _MIX1
        z = (z ^ (z >> _U64(27))) * _MIX2
        return z ^ (z >> _U64(31))


def normal_deviates(seed: int, stream: int, n_sites: int, n_mu: int) -> np.ndarray:
    """Standard normal deviates r[s, mu, a], a = 0..7, shape (n_sites, n_mu, 8).

    Counter key ``k = (((seed*4 + stream)*n_sites + s)*n_mu + mu)*8 + a``;
    uniforms ``u1 = (h(2k) >> 11 + 1) / 2^53`` in (0, 1] and
    ``u2 = (h(2k+1) >> 11) / 2^53`` in [0, 1); ``r = sqrt(-2 ln u1) cos(2 pi u2)``.
    """
    if not (0 <= stream < 4):
        raise ValueError("stream must be in 0..3")
    base = ((int(seed) * 4 + int(stream)) * int(n_sites)) * int(n_mu) * 8
    k = _U64(base) + np.arange(n_sites * n_mu * 8, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h1 = _splitmix64(k * _U64(2))
        h2 = _splitmix64(k * _U64(2) + _U64(1))
    u1 = ((h1 >> _U64(11)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = (h2 >> _U64(11)).astype(np.float64) * 2.0**-53
    r = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return r.reshape(n_sites, n_mu, 8)


def su3_from_coefficients(r: np.ndarray, scale: float) -> np.ndarray:
    """exp(i * scale * sum_a r_a lambda_a / 2) for r of shape (..., 8)."""
    lam = gell_mann()
    H = np.einsum("...a,aij->...ij", r * (0.5 * scale), lam)
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    w, v = np.linalg.eigh(H)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def random_links(L, seed: int, scale: float) -> np.ndarray:
    """Links U_mu(x) = exp(i scale sum r lambda/2), shape lattice_shape(L)+(4,3,3)."""
    shp = lattice_shape(L)
    V = int(np.prod(shp))
    r = normal_deviates(seed, 0, V, 4)
    return su3_from_coefficients(r, scale).reshape(shp + (4, 3, 3))


def random_gauge(L, seed: int, scale: float) -> np.ndarray:
    """Gauge transformation g(x), shape lattice_shape(L)+(3,3) (stream 1, mu = 0)."""
    shp = lattice_shape(L)
    V = int(np.prod(shp))
    r = normal_deviates(seed, 1, V, 1)[:, 0, :]
    return su3_from_coefficients(r, scale).reshape(shp + (3, 3))


# array axis of each lattice direction mu (x is the last lattice axis)
_AXIS = (3, 2, 1, 0)


def apply_gauge(U: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) <- g(x) U_mu(x) g(x+mu)^dagger (input preparation only)."""
    out = np.empty_like(U)
    gd = np.conj(np.swapaxes(g, -1, -2))
    for mu in range(4):
        gd_fwd = np.roll(gd, -1, axis=_AXIS[mu])
        out[..., mu, :, :] = np.einsum("...ij,...jk,...kl->...il", g, U[..., mu, :, :], gd_fwd)
    return out


def synthetic_config(L, seed: int, link_scale: float, gauge_scale: float = 1.0) -> np.ndarray:
    """Random links of ``link_scale`` hidden behind a random gauge of ``gauge_scale``."""
    U = random_links(L, seed, link_scale)
    if gauge_scale == 0.0:
        return U
    g = random_gauge(L, seed, gauge_scale)
    return apply_gauge(U, g)
