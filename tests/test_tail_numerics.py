"""The arithmetic of the double-float tail step, emulated in numpy float32
on the CPU: each operation rounded to nearest, and a fused multiply-add
(``_fma``) rounded once wherever the kernels use ``__fmaf_rn``, in the
kernels' order of operations.

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


def _fma(x, y, z):
    """FP32 fma(x, y, z) = x y + z rounded once to nearest (even).  The
    product of two FP32 numbers is exact in float64; the float64 sum s and
    its exact two-sum residual e settle the one case where rounding s to
    FP32 differs from rounding the exact value: s on an FP32 midpoint."""
    x, y, z = float(F(x)), float(F(y)), float(F(z))
    p = x * y
    s = p + z
    bb = s - p
    e = (p - (s - bb)) + (z - bb)
    r = F(s)
    if e != 0.0 and float(r) != s:
        dn = r if float(r) < s else np.nextafter(r, F(-np.inf))
        up = np.nextafter(r, F(np.inf)) if float(r) < s else r
        if s == (float(dn) + float(up)) / 2:
            r = up if e > 0 else dn
    return F(r)


def test_fma_emulation_rounds_once():
    """_fma against exact rational arithmetic, including products whose sum
    lands on an FP32 rounding midpoint after the float64 addition."""
    from fractions import Fraction
    rng = np.random.default_rng(2)

    def round32(q):
        # nearest FP32 to the rational q (ties to even), by bracketing
        f = F(float(q))
        lo = f if Fraction(float(f)) <= q else np.nextafter(f, F(-np.inf))
        hi = np.nextafter(lo, F(np.inf))
        dl, dh = q - Fraction(float(lo)), Fraction(float(hi)) - q
        if dl < dh:
            return lo
        if dh < dl:
            return hi
        return lo if (np.array([lo], F).view(np.uint32)[0] & 1) == 0 else hi

    cases = [(F(1 + 2.0 ** -12), F(1 + 2.0 ** -12), F(-(2.0 ** -24) * 0.5))]
    for _ in range(3000):
        x, y = F(rng.uniform(-2, 2)), F(rng.uniform(-2, 2))
        z = F(-float(x) * float(y) + rng.uniform(-1, 1) * 2.0 ** -rng.integers(0, 40))
        cases.append((x, y, z))
    for x, y, z in cases:
        exact = Fraction(float(x)) * Fraction(float(y)) + Fraction(float(z))
        assert _fma(x, y, z) == round32(exact)


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
    vfma = np.vectorize(_fma, otypes=[F])
    dl = vfma(nh, tl, vfma(nl, th, ml))
    d = (dh + dl).astype(F)
    ph, pl = _two_prod(y, (F(-0.5) * dh).astype(F))
    rest = vfma(y, vfma((F(0.375) * d).astype(F), d, (F(-0.5) * dl).astype(F)), pl)
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


# ---------------------------------------------------------------------------
# k_promote_df: Gram-Schmidt of the FP32 gauge G in double-float
# ---------------------------------------------------------------------------
class _Acc:
    """dacc: h advances by exact two-sums, every error into one FP32 l."""

    def __init__(self, h=0.0, lo=0.0):
        self.h, self.l = F(h), F(lo)

    def prod(self, x, y):  # x, y FP32
        p, e = _two_prod(np.array([x], F), np.array([y], F))
        s, t = _two_sum(np.array([self.h], F), p)
        self.h, self.l = s[0], F(self.l + F(e[0] + t[0]))

    def prod_df(self, xh, xl, y):  # x double-float, y FP32
        p, e = _two_prod(np.array([xh], F), np.array([y], F))
        s, t = _two_sum(np.array([self.h], F), p)
        self.h, self.l = s[0], F(self.l + F(_fma(xl, y, e[0]) + t[0]))

    def prod_dd(self, xh, xl, yh, yl):  # both double-float
        p, e = _two_prod(np.array([xh], F), np.array([yh], F))
        s, t = _two_sum(np.array([self.h], F), p)
        self.h, self.l = s[0], F(self.l + F(_fma(xh, yl, _fma(xl, yh, e[0])) + t[0]))

    def lo(self, x, y):  # dacc_lo: a first-order term into the low part, one FMA
        self.l = _fma(x, y, self.l)

    def result(self):
        s, e = _fast_two_sum(np.array([self.h], F), np.array([self.l], F))
        return s[0], e[0]


def _rsqrt_df(nh, nl):
    y = F(1.0 / np.sqrt(np.float64(nh)))
    th, tl = _two_prod(np.array([y], F), np.array([y], F))
    mh, ml = _two_prod(np.array([nh], F), th)
    dh = F(mh[0] - F(1.0))
    dl = _fma(nh, tl[0], _fma(nl, th[0], ml[0]))
    d = F(dh + dl)
    ph, pl = _two_prod(np.array([y], F), np.array([F(F(-0.5) * dh)], F))
    rest = _fma(y, _fma(F(F(0.375) * d), d, F(F(-0.5) * dl)), pl[0])
    qh, ql = _fast_two_sum(np.array([y], F), ph)
    return _fast_two_sum(qh, np.array([F(ql[0] + rest)], F))


def _mul_f(xh, xl, f):  # df_mul_f
    p, e = _two_prod(np.array([xh], F), np.array([f], F))
    return _fast_two_sum(p, np.array([_fma(xl, f, e[0])], F))


def _mul_dd(xh, xl, yh, yl):  # df_mul
    p, e = _two_prod(np.array([xh], F), np.array([yh], F))
    return _fast_two_sum(p, np.array([_fma(xh, yl, _fma(xl, yh, e[0]))], F))


def _promote(G):
    """Rows 0 and 1 of an FP32 3x3 complex G -> (Gh, Gl) in the kernel's order."""
    r0, r1 = G[0], G[1]
    n = _Acc()
    for j in range(3):
        n.prod(r0[j].real, r0[j].real)
        n.prod(r0[j].imag, r0[j].imag)
    ih, il = _rsqrt_df(*n.result())
    u = []
    for j in range(3):
        a = _mul_f(ih[0], il[0], r0[j].real)
        b = _mul_f(ih[0], il[0], r0[j].imag)
        u.append((a[0][0], a[1][0], b[0][0], b[1][0]))  # re h, re l, im h, im l
    pr, pi = _Acc(), _Acc()
    for j in range(3):
        urh, url, uih, uil = u[j]
        pr.prod_df(urh, url, r1[j].real)
        pr.prod_df(uih, uil, r1[j].imag)
        pi.prod_df(urh, url, r1[j].imag)
        pi.prod_df(-uih, -uil, r1[j].real)
    ipr, ipi = pr.result(), pi.result()
    w = []
    for j in range(3):
        urh, url, uih, uil = u[j]
        a, b = _Acc(r1[j].real), _Acc(r1[j].imag)
        a.prod_dd(-ipr[0], -ipr[1], urh, url)
        a.prod_dd(ipi[0], ipi[1], uih, uil)
        b.prod_dd(-ipr[0], -ipr[1], uih, uil)
        b.prod_dd(-ipi[0], -ipi[1], urh, url)
        w.append(a.result() + b.result())
    n = _Acc()
    for j in range(3):
        n.prod_dd(w[j][0], w[j][1], w[j][0], w[j][1])
        n.prod_dd(w[j][2], w[j][3], w[j][2], w[j][3])
    jh, jl = _rsqrt_df(*n.result())
    w2 = []
    for j in range(3):
        a = _mul_dd(w[j][0], w[j][1], jh[0], jl[0])
        b = _mul_dd(w[j][2], w[j][3], jh[0], jl[0])
        w2.append((a[0][0], a[1][0], b[0][0], b[1][0]))
    v = []
    for j in range(3):
        k, l = (j + 1) % 3, (j + 2) % 3
        ukr, ukrl, uki, ukil = u[k]
        ulr, ulrl, uli, ulil = u[l]
        wkr, wkrl, wki, wkil = w2[k]
        wlr, wlrl, wli, wlil = w2[l]
        a, b = _Acc(), _Acc()
        a.prod_dd(ukr, ukrl, wlr, wlrl)
        a.prod_dd(-uki, -ukil, wli, wlil)
        a.prod_dd(-ulr, -ulrl, wkr, wkrl)
        a.prod_dd(uli, ulil, wki, wkil)
        b.prod_dd(-ukr, -ukrl, wli, wlil)
        b.prod_dd(-uki, -ukil, wlr, wlrl)
        b.prod_dd(ulr, ulrl, wki, wkil)
        b.prod_dd(uli, ulil, wkr, wkrl)
        v.append(a.result() + b.result())
    M = np.zeros((3, 3), np.complex128)
    for j in range(3):
        for row, src in ((0, u[j]), (1, w2[j]), (2, v[j])):
            M[row, j] = (np.float64(src[0]) + np.float64(src[1])) + 1j * (np.float64(src[2]) + np.float64(src[3]))
    return M


def test_double_float_promote_is_special_unitary_to_double_float_accuracy():
    """k_promote_df's Gram-Schmidt, emulated: for FP32 gauge matrices within
    ~1e-6 of SU(3), Gh + Gl is unitary with det 1 to ~2^-46, and rows 0 and 1
    span the same directions as the input's (it reunitarises, it does not
    move the matrix)."""
    rng = np.random.default_rng(9)
    worst = 0.0
    for _ in range(200):
        A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        Q, R = np.linalg.qr(A)
        Q = Q * (np.diag(R) / np.abs(np.diag(R)))
        Q[2] = np.conj(np.cross(Q[0], Q[1]))  # SU(3)
        G = (Q + 1e-6 * (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))).astype(np.complex64)
        M = _promote(G)
        worst = max(worst, np.max(np.abs(M @ M.conj().T - np.eye(3))), abs(np.linalg.det(M) - 1))
        # row 0 is G's row 0 normalised
        r0 = G[0].astype(np.complex128)
        assert np.max(np.abs(M[0] - r0 / np.linalg.norm(r0))) < 1e-14
    assert worst < 2.0 ** -45


# ---------------------------------------------------------------------------
# k_tail_start_df: U = g U_loaded g'^dag in double-float
# ---------------------------------------------------------------------------
def _split64(x):
    """split_fp64: hi = x truncated to 24 significant bits, lo = the rest
    rounded to FP32."""
    b = np.array([x], np.float64).view(np.uint64)[0]
    hi = np.array([b & np.uint64(0xFFFFFFFFE0000000)], np.uint64).view(np.float64)[0]
    return F(hi), F(x - hi)


def _tail_link(gh, gl, U, fh, fl):
    """One link, rows of W = g U with the first-order terms in the low parts,
    then W f^dag likewise (the kernel's order)."""
    UH = np.zeros((3, 3), np.complex64)
    UL = np.zeros((3, 3), np.complex64)
    for i in range(3):
        for j in range(3):
            rh, rl = _split64(U[i, j].real)
            ih, il = _split64(U[i, j].imag)
            UH[i, j], UL[i, j] = complex(rh, ih), complex(rl, il)
    out = np.zeros((3, 3), np.complex128)
    for a in range(3):
        W = []
        for b in range(3):
            re, im = _Acc(), _Acc()
            for k in range(3):
                x, y, xe, ye = gh[a, k], UH[k, b], gl[a, k], UL[k, b]
                re.prod(x.real, y.real)
                re.prod(-x.imag, y.imag)
                im.prod(x.real, y.imag)
                im.prod(x.imag, y.real)
                re.lo(xe.real, y.real)
                re.lo(-xe.imag, y.imag)
                re.lo(x.real, ye.real)
                re.lo(-x.imag, ye.imag)
                im.lo(xe.real, y.imag)
                im.lo(xe.imag, y.real)
                im.lo(x.real, ye.imag)
                im.lo(x.imag, ye.real)
            W.append(re.result() + im.result())
        for b in range(3):
            re, im = _Acc(), _Acc()
            for k in range(3):
                wrh, wrl, wih, wil = W[k]
                f, fe = fh[b, k], fl[b, k]
                re.prod_df(wrh, wrl, f.real)
                re.prod_df(wih, wil, f.imag)
                im.prod_df(wih, wil, f.real)
                im.prod_df(-wrh, -wrl, f.imag)
                re.lo(wrh, fe.real)
                re.lo(wih, fe.imag)
                im.lo(wih, fe.real)
                im.lo(-wrh, fe.imag)
            rh, rl = re.result()
            ih, il = im.result()
            out[a, b] = (np.float64(rh) + np.float64(rl)) + 1j * (np.float64(ih) + np.float64(il))
    return out


def _split_df(M):
    h = M.astype(np.complex64)
    return h, (M - h.astype(np.complex128)).astype(np.complex64)


def test_double_float_tail_start_forms_the_link_to_double_float_accuracy():
    """k_tail_start_df, emulated: with g, g' double-float matrices and U an
    FP64 SU(3) link, g U g'^dag comes out within ~2^-46 of the product in
    FP64 (the dropped second-order terms and the roundings are ~2^-48 each)."""
    rng = np.random.default_rng(13)

    def su3():
        A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        Q, R = np.linalg.qr(A)
        Q = Q * (np.diag(R) / np.abs(np.diag(R)))
        Q[2] = np.conj(np.cross(Q[0], Q[1]))
        return Q

    worst_err = 0.0
    for _ in range(100):
        g, U, f = su3(), su3(), su3()
        gh, gl = _split_df(g)
        fh, fl = _split_df(f)
        gd = gh.astype(np.complex128) + gl.astype(np.complex128)
        fd = fh.astype(np.complex128) + fl.astype(np.complex128)
        ref = gd @ U @ fd.conj().T
        got = _tail_link(gh, gl, U, fh, fl)
        worst_err = max(worst_err, np.max(np.abs(got - ref)))
    assert worst_err < 2.0 ** -45
