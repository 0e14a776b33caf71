"""Pins of the CPU oracle against facts that do not come from the oracle:
closed forms derived from the definitions of the method (Sec. 1 of the paper,
steepest descent with Fourier acceleration), library routines (numpy FFT, QR,
scipy expm), brute force on tiny lattices, finite differences and invariants.

Each test names the mistake it is there to catch.
"""
import json
import math
import os

import numpy as np
import pytest

import lgf_inputs as I
from oracle import lgf_oracle as O

from . import brute_force as BF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 0.08


def _abelian_links(omega, H=(1.0, -1.0, 0.0)):
    """U_mu(x) = exp(i (omega(x) - omega(x+mu)) H): pure gauge, diagonal."""
    shp = omega.shape
    U = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        phi = omega - np.roll(omega, -1, axis=O.AXIS[mu])
        for j in range(3):
            U[..., mu, j, j] = np.exp(1j * phi * H[j])
    return U


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def test_generator_is_su3_and_seeded():
    U = I.synthetic_config((4, 3, 2, 5), seed=7, link_scale=0.6)
    assert O.unitarity_defect(U) < 1e-13
    U2 = I.synthetic_config((4, 3, 2, 5), seed=7, link_scale=0.6)
    assert np.array_equal(U, U2)
    U3 = I.synthetic_config((4, 3, 2, 5), seed=8, link_scale=0.6)
    assert np.max(np.abs(U - U3)) > 0.1


def test_normal_deviates_moments():
    r = I.normal_deviates(3, 0, 4096, 4).ravel()
    assert abs(r.mean()) < 0.02 and abs(r.var() - 1.0) < 0.03
    assert abs(np.mean(r ** 4) - 3.0) < 0.15


# ---------------------------------------------------------------------------
# SU(3) projection and exponential
# ---------------------------------------------------------------------------

def test_reunitarize_matches_qr():
    """Gram-Schmidt on rows 1, 2 == QR of their transpose with positive R
    diagonal; row 3 completes det = +1.  Catches a wrong inner-product
    conjugation or a wrong cross-product sign."""
    rng = np.random.default_rng(0)
    M = rng.standard_normal((50, 3, 3)) + 1j * rng.standard_normal((50, 3, 3))
    R = O.reunitarize(M)
    assert O.unitarity_defect(R) < 1e-13
    for n in range(50):
        q, r = np.linalg.qr(M[n, :2, :].T)
        q = q * (np.diag(r) / np.abs(np.diag(r))).conj()[None, :]  # positive diagonal
        np.testing.assert_allclose(R[n, :2, :], q.T, atol=1e-13)
        np.testing.assert_allclose(np.linalg.det(R[n]), 1.0, atol=1e-13)


def test_reunitarize_fixes_su3():
    U = I.random_links((2, 2, 2, 2), 1, 1.0)
    np.testing.assert_allclose(O.reunitarize(U), U, atol=1e-14)


def test_exact_exponential_matches_scipy():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(2)
    A = rng.standard_normal((20, 3, 3)) + 1j * rng.standard_normal((20, 3, 3))
    X = A - O.dagger(A)
    E = O.expm_antihermitian(X)
    for n in range(20):
        np.testing.assert_allclose(E[n], scipy_linalg.expm(X[n]), atol=1e-12)


# ---------------------------------------------------------------------------
# Fourier transform and momentum factor
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 2, 4, 5)])
def test_dft_matches_bruteforce_and_numpy(dims):
    rng = np.random.default_rng(3)
    shp = I.lattice_shape(dims)
    f = rng.standard_normal(shp + (2,)) + 1j * rng.standard_normal(shp + (2,))
    fk = O.dft4(f, -1)
    # brute force V x V sum
    Lx, Ly, Lz, Lt = dims
    pts = [(t, z, y, x) for t in range(Lt) for z in range(Lz) for y in range(Ly) for x in range(Lx)]
    for k in pts[:: max(1, len(pts) // 13)]:
        acc = np.zeros(2, dtype=np.complex128)
        for c in pts:
            ph = sum(k[a] * c[a] / shp[a] for a in range(4))
            acc += f[c] * np.exp(-2j * np.pi * ph)
        np.testing.assert_allclose(fk[k], acc, atol=1e-12)
    # textbook library routine (forward e^{-}, unnormalised)
    np.testing.assert_allclose(fk, np.fft.fftn(f, axes=(0, 1, 2, 3)), atol=1e-11)
    # inverse with 1/V returns the input; Parseval
    V = f[..., 0].size
    np.testing.assert_allclose(O.dft4(fk, +1) / V, f, atol=1e-12)
    assert abs(np.sum(np.abs(fk) ** 2) / V - np.sum(np.abs(f) ** 2)) < 1e-10


def test_plane_wave_maps_to_one_mode():
    dims = (4, 6, 2, 8)
    shp = I.lattice_shape(dims)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in shp], indexing="ij")
    k = (3, 1, 5, 2)  # (kt, kz, ky, kx)
    f = np.exp(2j * np.pi * (k[0] * t / 8 + k[1] * z / 2 + k[2] * y / 6 + k[3] * x / 4))
    fk = O.dft4(f, -1)
    V = f.size
    expect = np.zeros(shp, dtype=np.complex128)
    expect[k] = V
    np.testing.assert_allclose(fk, expect, atol=1e-10)


def test_momentum_on_2_4():
    """On 2^4, p2 = 4 * (number of odd k components): 0,4,...,16 with
    binomial multiplicities; p2_max = 16."""
    p2 = O.momentum_sq((2, 2, 2, 2))
    vals, counts = np.unique(np.round(p2, 12), return_counts=True)
    np.testing.assert_allclose(vals, [0, 4, 8, 12, 16], atol=1e-12)
    assert list(counts) == [1, 4, 6, 4, 1]
    assert O.p2_max((2, 2, 2, 2)) == pytest.approx(16.0, abs=1e-12)
    for dims in [(8, 8, 8, 8), (32, 32, 32, 32), (48, 48, 48, 8), (24, 24, 24, 48), (20, 20, 20, 20)]:
        assert O.p2_max(dims) == pytest.approx(16.0, abs=1e-12)
    assert O.p2_max((3, 3, 3, 3)) == pytest.approx(4 * 4 * math.sin(math.pi / 3) ** 2)


# ---------------------------------------------------------------------------
# gradient, F, theta
# ---------------------------------------------------------------------------

def test_single_link_closed_form():
    gold = json.load(open(os.path.join(GOLDEN, "single_link.json")))
    for phi in gold["phis"]:
        U = np.broadcast_to(np.eye(3, dtype=np.complex128), (2, 2, 2, 2, 4, 3, 3)).copy()
        U[0, 0, 0, 0, 0] = np.diag([np.exp(1j * phi), np.exp(-1j * phi), 1.0])
        D = O.gradient(U)
        F, theta = O.functional(U, D)
        assert theta == pytest.approx(math.sin(phi) ** 2 / 3, rel=1e-14)
        assert F == pytest.approx((190 + 2 * math.cos(phi)) / 192, rel=1e-14)
        np.testing.assert_allclose(np.diag(D[0, 0, 0, 0]).imag,
                                   [-2 * math.sin(phi), 2 * math.sin(phi), 0], atol=1e-15)
        np.testing.assert_allclose(np.diag(D[0, 0, 0, 1]).imag,
                                   [2 * math.sin(phi), -2 * math.sin(phi), 0], atol=1e-15)
        others = np.abs(D).sum(axis=(-2, -1))
        others[0, 0, 0, 0] = others[0, 0, 0, 1] = 0
        assert others.max() == 0


def test_gradient_is_derivative_of_functional():
    """dF/d eps of F(U^{exp(eps X) at one site}) = <X, Delta(x)> / (2 N_d N_c V).
    Catches a wrong sign, a missing factor or a shift in the wrong direction."""
    dims = (3, 4, 2, 5)
    U = I.synthetic_config(dims, seed=11, link_scale=0.7)
    D = O.gradient(U)
    V = np.prod(dims)
    rng = np.random.default_rng(4)
    shp = I.lattice_shape(dims)
    for trial in range(4):
        site = tuple(rng.integers(0, n) for n in shp)
        A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        X = A - A.conj().T
        X -= np.trace(X) / 3 * np.eye(3)
        eps = 1e-5
        vals = []
        for s in (+1, -1):
            g = np.broadcast_to(np.eye(3, dtype=np.complex128), shp + (3, 3)).copy()
            g[site] = O.expm_antihermitian(s * eps * X[None])[0]
            vals.append(O.functional(O.gauge_transform(U, g))[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        expect = np.real(np.trace(X.conj().T @ D[site])) / (2 * 12 * V)
        assert fd == pytest.approx(expect, rel=1e-6, abs=1e-12)


def test_zero_momentum_mode_is_roundoff():
    U = I.synthetic_config((4, 4, 4, 4), seed=5, link_scale=0.5)
    D = O.gradient(U)
    assert np.max(np.abs(D.sum(axis=(0, 1, 2, 3)))) < 1e-12 * D.size
    a = O.accelerate(D, zero_mode=0.0)
    b = O.accelerate(D, zero_mode=1.0)
    assert np.max(np.abs(a - b)) < 1e-13


# ---------------------------------------------------------------------------
# closed forms of the whole iteration
# ---------------------------------------------------------------------------

def test_linearised_abelian_rate_with_acceleration():
    """Pure abelian gauge, amplitude 1e-6: every mode shrinks by (1 - alpha
    p2_max), so theta_{n+1}/theta_n = (1 - 16 alpha)^2 = 0.0784.  Pins the
    sign of Delta, alpha/2, the momentum factor and the 1/V normalisation."""
    rng = np.random.default_rng(1)
    omega = 1e-6 * rng.standard_normal(I.lattice_shape((4, 6, 4, 8)))
    hist = []
    O.iterate(_abelian_links(omega), 4, ALPHA, history=hist)
    for a, b in zip(hist[:-1], hist[1:]):
        assert b[1] / a[1] == pytest.approx((1 - 16 * ALPHA) ** 2, rel=1e-8)


@pytest.mark.parametrize("k", [(1, 0, 0, 0), (0, 2, 0, 1), (2, 3, 1, 3)])
def test_linearised_abelian_plane_wave_without_acceleration(k):
    """Without acceleration a plane wave k shrinks by (1 - alpha p2(k))."""
    dims = (4, 6, 2, 8)
    shp = I.lattice_shape(dims)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in shp], indexing="ij")
    kx, ky, kz, kt = k
    omega = 1e-6 * np.cos(2 * np.pi * (kx * x / 4 + ky * y / 6 + kz * z / 2 + kt * t / 8))
    p2 = sum(4 * math.sin(math.pi * kk / n) ** 2 for kk, n in zip(k, dims))
    hist = []
    O.iterate(_abelian_links(omega), 3, ALPHA, accel=False, history=hist)
    for a, b in zip(hist[:-1], hist[1:]):
        assert b[1] / a[1] == pytest.approx((1 - ALPHA * p2) ** 2, rel=1e-7)


def test_constant_links_are_fixed_points():
    u = I.random_links((1, 1, 1, 1), 9, 1.3)[0, 0, 0, 0]  # 4 random SU(3)
    U = np.broadcast_to(u, (3, 2, 4, 2, 4, 3, 3)).copy()
    D = O.gradient(U)
    assert np.max(np.abs(D)) < 1e-15
    assert O.functional(U, D)[1] < 1e-30
    np.testing.assert_allclose(O.iterate(U, 1, ALPHA), U, atol=1e-15)


def test_pure_gauge_fixes_to_unit_links():
    dims = (4, 2, 3, 4)
    g = I.random_gauge(dims, 3, 0.3)
    U = I.apply_gauge(np.broadcast_to(np.eye(3, dtype=np.complex128),
                                      I.lattice_shape(dims) + (4, 3, 3)).copy(), g)
    r = O.fix(U, 1e-26, 500, ALPHA)
    assert r["converged"]
    assert r["F"] == pytest.approx(1.0, abs=1e-14)
    assert np.max(np.abs(r["U"] - np.eye(3))) < 1e-11


# ---------------------------------------------------------------------------
# invariants and brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("exp_order", [1, 0])
def test_invariants_along_the_run(exp_order):
    U0 = I.synthetic_config((4, 4, 4, 6), seed=0, link_scale=0.5)
    plaq0 = O.average_plaquette(U0)
    r = O.fix(U0, 1e-14, 300, ALPHA, exp_order=exp_order, track_gauge=True)
    assert r["converged"]
    Fs = [h[0] for h in r["history"]]
    assert all(b >= a - 1e-15 * abs(a) for a, b in zip(Fs[:-1], Fs[1:]))
    assert O.unitarity_defect(r["U"]) < 1e-13
    assert O.unitarity_defect(r["G"]) < 1e-13
    assert O.average_plaquette(r["U"]) == pytest.approx(plaq0, abs=1e-13)
    # the tracked transformation reproduces the final links from the start
    np.testing.assert_allclose(O.gauge_transform(U0, r["G"]), r["U"], atol=1e-12)


def test_converged_gauge_is_local_maximum():
    U0 = I.synthetic_config((4, 4, 4, 4), seed=2, link_scale=0.5)
    r = O.fix(U0, 1e-24, 500, ALPHA)
    assert r["converged"]
    rng = np.random.default_rng(6)
    shp = r["U"].shape[:4]
    for _ in range(20):
        A = rng.standard_normal(shp + (3, 3)) + 1j * rng.standard_normal(shp + (3, 3))
        X = 1e-4 * (A - O.dagger(A))
        g = O.expm_antihermitian(X)
        assert O.functional(O.gauge_transform(r["U"], g))[0] < r["F"]


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 2, 4, 2)])
def test_oracle_matches_brute_force(dims):
    U = I.synthetic_config(dims, seed=4, link_scale=0.8)
    links, L = BF.from_array(U)
    Uo = U
    for _ in range(3):
        links, Fb, thb = BF.one_iteration(links, L, ALPHA)
        hist = []
        Uo = O.iterate(Uo, 1, ALPHA, history=hist)
        assert hist[0][0] == pytest.approx(Fb, rel=1e-13)
        assert hist[0][1] == pytest.approx(thb, rel=1e-12)
        assert BF.max_diff(links, Uo) < 1e-13


def test_pack_delta_holds_the_eight_real_degrees_of_freedom():
    """pack_delta (the 4-complex packing the GPU's gradient planes use): a
    traceless anti-Hermitian matrix is X = i sum_a c_a lambda_a / 2, built here
    from the Gell-Mann matrices with known c_a; its packed form must hold
    X01, X02, X12 and Im X00 + i Im X11 (closed forms in the c_a checked too),
    so a wrong index, sign or conjugate in the packing fails.  Unpacking the
    4 numbers by the anti-Hermitian, traceless rules rebuilds X exactly."""
    rng = np.random.default_rng(31)
    lam = I.gell_mann()
    c = rng.normal(size=(5, 8))
    X = np.einsum("na,aij->nij", 0.5j * c, lam)
    P = O.pack_delta(X)
    assert P.shape == (5, 4)
    for n in range(5):
        x00, x11 = X[n, 0, 0].imag, X[n, 1, 1].imag
        assert P[n, 0] == X[n, 0, 1] and P[n, 1] == X[n, 0, 2] and P[n, 2] == X[n, 1, 2]
        assert P[n, 3] == x00 + 1j * x11
        # closed forms of the entries from the coefficients
        assert np.isclose(X[n, 0, 1], 0.5j * (c[n, 0] - 1j * c[n, 1]))
        assert np.isclose(x00, 0.5 * (c[n, 2] + c[n, 7] / math.sqrt(3)))
        # rebuild from the 4 numbers
        R = np.zeros((3, 3), complex)
        R[0, 1], R[0, 2], R[1, 2] = P[n, 0], P[n, 1], P[n, 2]
        R[1, 0], R[2, 0], R[2, 1] = -np.conj(P[n, 0]), -np.conj(P[n, 1]), -np.conj(P[n, 2])
        R[0, 0], R[1, 1] = 1j * P[n, 3].real, 1j * P[n, 3].imag
        R[2, 2] = -1j * (P[n, 3].real + P[n, 3].imag)
        assert np.allclose(R, X[n], atol=1e-15)
