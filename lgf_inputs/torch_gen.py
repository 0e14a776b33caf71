"""The synthetic-configuration recipe of ``lgf_inputs`` computed with torch on
a GPU, for lattices too large to generate quickly on the host (the batched
benchmark holds 64 lattices, 18.4 million sites).

Same counters, same Box-Muller deviates and same matrices as the numpy
generator, up to rounding: the deviates agree to a few ulp (the device's log
and cos differ in the last bits from the host's), and the exponential is a
Taylor series with scaling and squaring instead of an eigen-decomposition
(agreement ~1e-15; the result is unitary with unit determinant to rounding).
Holds none of the gauge-fixing method's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gell_mann, lattice_shape

# SplitMix64 constants as two's-complement int64 (torch has no uint64 math)
_GOLDEN = 0x9E3779B97F4A7C15 - (1 << 64)
_MIX1 = 0xBF58476D1CE4E5B9 - (1 << 64)
_MIX2 = 0x94D049BB133111EB - (1 << 64)


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _splitmix64(z: torch.Tensor) -> torch.Tensor:
    z = z + _GOLDEN
    z = (z ^ _srl(z, 30)) * _MIX1
    z = (z ^ _srl(z, 27)) * _MIX2
    return z ^ _srl(z, 31)


def normal_deviates(seed: int, stream: int, n_sites: int, n_mu: int, device) -> torch.Tensor:
    """r[s, mu, a] as in lgf_inputs.normal_deviates, float64 on `device`."""
    base = ((int(seed) * 4 + int(stream)) * int(n_sites)) * int(n_mu) * 8
    if base >= (1 << 62):
        raise ValueError("counter out of range")
    k = base + torch.arange(n_sites * n_mu * 8, dtype=torch.int64, device=device)
    h1 = _splitmix64(k * 2)
    h2 = _splitmix64(k * 2 + 1)
    u1 = (_srl(h1, 11).to(torch.float64) + 1.0) * 2.0 ** -53
    u2 = _srl(h2, 11).to(torch.float64) * 2.0 ** -53
    r = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    return r.reshape(n_sites, n_mu, 8)


def _mm(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return (a.unsqueeze(-1) * b.unsqueeze(-3)).sum(-2)


def _expi(H: torch.Tensor) -> torch.Tensor:
    """exp(iH) for Hermitian 3x3 H: Taylor series of degree 16 after scaling
    by 2^-s so that the norm is below 1/4, then s squarings."""
    X = 1j * H
    nrm = torch.linalg.matrix_norm(X, ord="fro").max().item()
    s = max(0, int(math.ceil(math.log2(max(nrm, 1e-300) / 0.25)))) if nrm > 0.25 else 0
    X = X / (2.0 ** s)
    eye = torch.eye(3, dtype=X.dtype, device=X.device).expand_as(X)
    E = eye.clone()
    for k in range(16, 0, -1):  # Horner: I + X/1 (I + X/2 (I + ...))
        E = eye + _mm(X, E) / k
    for _ in range(s):
        E = _mm(E, E)
    return E


def su3_from_coefficients(r: torch.Tensor, scale: float) -> torch.Tensor:
    lam = torch.from_numpy(gell_mann()).to(r.device)
    H = torch.einsum("...a,aij->...ij", (r * (0.5 * scale)).to(torch.complex128), lam)
    H = 0.5 * (H + H.conj().transpose(-1, -2))
    return _expi(H)


_AXIS = (3, 2, 1, 0)


def synthetic_config(L, seed: int, link_scale: float, gauge_scale: float = 1.0, device="cuda",
                     chunk: int = 1 << 20) -> torch.Tensor:
    """complex128 tensor (Lt, Lz, Ly, Lx, 4, 3, 3) on `device`, the recipe of
    lgf_inputs.synthetic_config."""
    shp = lattice_shape(L)
    V = int(np.prod(shp))
    U = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device=device)
    r_all = normal_deviates(seed, 0, V, 4, device)
    for a in range(0, V, chunk):
        U[a:a + chunk] = su3_from_coefficients(r_all[a:a + chunk], link_scale)
    del r_all
    U = U.reshape(shp + (4, 3, 3))
    if gauge_scale == 0.0:
        return U
    r = normal_deviates(seed, 1, V, 1, device)[:, 0, :]
    g = torch.empty((V, 3, 3), dtype=torch.complex128, device=device)
    for a in range(0, V, chunk):
        g[a:a + chunk] = su3_from_coefficients(r[a:a + chunk], gauge_scale)
    g = g.reshape(shp + (3, 3))
    gd = g.conj().transpose(-1, -2)
    for mu in range(4):
        gdf = torch.roll(gd, shifts=-1, dims=_AXIS[mu])
        U[..., mu, :, :] = _mm(_mm(g, U[..., mu, :, :]), gdf)
    return U
