"""The arithmetic of the double-float tail step, emulated in numpy float32
(each operation rounded to nearest, no fused multiply-add), on the CPU.

The tail accumulates its gauge transformation 1 + eta <- (1 + eps)(1 + eta),
eps = X + X^2/2 with X = alpha/2 Delta~ traceless anti-Hermitian, |X| ~ 1e-5.
Stored in double-float (hi + lo), with X added by exact two-sums and only the
~|X|^2 Hermitian terms rounded in FP32, 1 + eta stays unitary to O(|X|^3)
(the second-order exponential's own error).  Rounding X + X^2/2 as one FP32
sum instead breaks unitarity by ~2^-24 |X| per step: that FP32-only form
ended one full-size fix with a unitarity defect of 1.3e-12.  These tests pin
both statements; the kernel that implements the first is k_tail_eta_step."""
import numpy as np

F = np.float32


def _two_sum(a, b):
    s = (a + b).astype(F)
    bb = (s - a).astype(F)
    e = ((a - (s - bb)).astype(F) + (b - bb).astype(F)).astype(F)
    return s, e


def _fast_two_sum(a, b):
    s = (a + b).astype(F)
    return s, (b - (s - a).astype(F)).astype(F)


def _mm32(a, b):
    """3x3 complex product with every real multiply and add rounded to FP32,
    in the order of the kernel's complex multiply-accumulate."""
    ar, ai, br, bi = a.real.astype(F), a.imag.astype(F), b.real.astype(F), b.imag.astype(F)
    cr = np.zeros((3, 3), F)
    ci = np.zeros((3, 3), F)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                cr[i, j] = F(F(cr[i, j] + F(ar[i, k] * br[k, j])) - F(ai[i, k] * bi[k, j]))
                ci[i, j] = F(F(ci[i, j] + F(ar[i, k] * bi[k, j])) + F(ai[i, k] * br[k, j]))
    return cr + 1j * ci


def _random_X(rng, size):
    """Traceless anti-Hermitian 3x3 with FP32 entries, X_ji = -conj(X_ij)
    exactly, as the kernel builds it from the packed gradient."""
    c = (rng.normal(size=4) + 1j * rng.normal(size=4)).astype(np.complex64) * F(size)
    X = np.zeros((3, 3), np.complex64)
    X[0, 0] = 1j * c[3].real
    X[1, 1] = 1j * c[3].imag
    X[2, 2] = -1j * F(c[3].real + c[3].imag)
    X[0, 1], X[0, 2], X[1, 2] = c[0], c[1], c[2]
    X[1, 0], X[2, 0], X[2, 1] = -np.conj(c[0]), -np.conj(c[1]), -np.conj(c[2])
    return X


def _step_double_float(eh, el, X):
    """eta <- eta + X + (X^2/2 + eps eta_hi): X by exact two-sums, the rest in FP32."""
    Y = (_mm32(X, X) * F(0.5)).astype(np.complex64)
    eps = (X + Y).astype(np.complex64)
    Y = (Y + _mm32(eps, eh)).astype(np.complex64)
    out_h = np.zeros((3, 3), np.complex64)
    out_l = np.zeros((3, 3), np.complex64)
    for part in ("real", "imag"):
        h = getattr(eh, part).astype(F)
        lo = getattr(el, part).astype(F)
        x = getattr(X, part).astype(F)
        y = getattr(Y, part).astype(F)
        s, e = _two_sum(h, x)
        s, e = _fast_two_sum(s, (e + (lo + y).astype(F)).astype(F))
        if part == "real":
            out_h.real, out_l.real = s, e
        else:
            out_h.imag, out_l.imag = s, e
    return out_h, out_l


def _step_fp32(e32, X):
    """The FP32-only form: eps = fl(X + X^2/2), eta <- fl(eta + eps + eps eta)."""
    eps = (X + (_mm32(X, X) * F(0.5)).astype(np.complex64)).astype(np.complex64)
    return (e32 + eps + _mm32(eps, e32)).astype(np.complex64)


def _defect(eta):
    H = np.eye(3) + eta.astype(np.complex128)
    return np.max(np.abs(H @ H.conj().T - np.eye(3)))


def test_double_float_step_keeps_the_gauge_transformation_unitary():
    rng = np.random.default_rng(7)
    worst_df = worst_fp32 = 0.0
    for trial in range(20):
        eh = np.zeros((3, 3), np.complex64)
        el = np.zeros((3, 3), np.complex64)
        e32 = np.zeros((3, 3), np.complex64)
        size = 4e-6
        for _ in range(5):  # the tail's steps shrink by ~4x each
            X = _random_X(rng, size)
            eh, el = _step_double_float(eh, el, X)
            e32 = _step_fp32(e32, X)
            size /= 4.0
        eta = eh.astype(np.complex128) + el.astype(np.complex128)
        worst_df = max(worst_df, _defect(eta))
        worst_fp32 = max(worst_fp32, _defect(e32))
    # O(|X|^3) ~ 1e-16 plus FP32 rounding of ~|X|^2 terms ~ 1e-18
    assert worst_df < 2e-15
    # the FP32-only form loses ~2^-24 |X| ~ 1e-13 at the first step
    assert worst_fp32 > 1e-14
    assert worst_fp32 > 20 * worst_df


def test_two_sum_is_exact():
    """Knuth's two-sum, as in lgf_df.cuh: s + e equals a + b exactly."""
    rng = np.random.default_rng(3)
    a = (rng.normal(size=10000) * np.exp(rng.normal(size=10000) * 5)).astype(F)
    b = (rng.normal(size=10000) * np.exp(rng.normal(size=10000) * 5)).astype(F)
    s, e = _two_sum(a, b)
    np.testing.assert_array_equal(s.astype(np.float64) + e.astype(np.float64),
                                  a.astype(np.float64) + b.astype(np.float64))


def _two_prod(a, b):
    """p + e = a b exactly: the FMA's exact residual, emulated in float64
    (a product of two FP32 numbers is exact in float64)."""
    p = (a * b).astype(F)
    e = (a.astype(np.float64) * b.astype(np.float64) - p.astype(np.float64)).astype(F)
    return p, e


def test_corrected_rsqrt_reaches_double_float_accuracy():
    """df_rsqrt: y = an approximate 1/sqrt(n.h) (here off by up to 4 ulp, as
    a hardware approximation may be), then with n y^2 = 1 + d formed exactly,
    1/sqrt(n) = y (1 - d/2 + 3 d^2/8): relative error ~2^-47, for n within
    1e-3 of 1 as the row norms of a nearly unitary matrix are.  The quadratic
    term takes the whole d = dh + dl: with dh^2 alone (an earlier form) the
    dropped 3/4 dh dl left ~2^-44."""
    rng = np.random.default_rng(11)
    nh = (1.0 + rng.uniform(-1e-3, 1e-3, 5000)).astype(F)
    nl = (rng.uniform(-1, 1, 5000) * np.spacing(nh) * 0.5).astype(F)
    exact = 1.0 / np.sqrt(nh.astype(np.longdouble) + nl.astype(np.longdouble))
    y = (1.0 / np.sqrt(nh.astype(np.float64))).astype(F)
    y = (y + rng.integers(-4, 5, 5000) * np.spacing(y)).astype(F)  # the approximation
    th, tl = _two_prod(y, y)
    mh, ml = _two_prod(nh, th)
    dh = (mh - F(1.0)).astype(F)  # exact (Sterbenz)
    dl = ((nh * tl).astype(F) + (nl * th).astype(F) + ml).astype(F)
    d = (dh + dl).astype(F)
    ph, pl = _two_prod(y, (F(-0.5) * dh).astype(F))
    rest = (y * ((F(0.375) * d).astype(F) * d - F(0.5) * dl).astype(F) + pl).astype(F)
    qh, ql = _fast_two_sum(y, ph)
    rh, rl = _fast_two_sum(qh, (ql + rest).astype(F))
    got = rh.astype(np.longdouble) + rl.astype(np.longdouble)
    rel = np.abs(got / exact - 1.0)
    assert float(np.max(rel)) < 2.0 ** -46
    # the uncorrected approximation is ~2^-21 off: the correction is what matters
    assert float(np.max(np.abs(y.astype(np.longdouble) / exact - 1.0))) > 2.0 ** -24


def test_dot2_accumulation_reaches_double_float_accuracy():
    """dacc_prod (Dot2): the running high part advances by exact two-sums and
    all product and sum errors go to one FP32 low part.  A 3-term complex dot
    product of FP32 numbers (6 real products) comes out accurate to ~2^-47 of
    the sum of |terms|."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(2000):
        x = rng.uniform(-1, 1, 6).astype(F)
        y = rng.uniform(-1, 1, 6).astype(F)
        h, lo = F(0.0), F(0.0)
        for a, b in zip(x, y):
            p, e = _two_prod(np.array([a]), np.array([b]))
            s, t = _two_sum(np.array([h]), p)
            h = s[0]
            lo = F(lo + F(e[0] + t[0]))
        got = np.longdouble(h) + np.longdouble(lo)
        exact = np.sum(x.astype(np.longdouble) * y.astype(np.longdouble))
        scale = np.sum(np.abs(x.astype(np.longdouble) * y.astype(np.longdouble)))
        worst = max(worst, float(abs(got - exact) / scale))
    assert worst < 2.0 ** -46
