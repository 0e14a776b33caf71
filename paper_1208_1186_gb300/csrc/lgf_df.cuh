// Double-float arithmetic on the FP32 pipe for the FP64 tail (value = h + l,
// |l| <= ulp(h)/2, 48 significant bits).  Built from the error-free
// transformations of Knuth (two-sum), Dekker (fast-two-sum) and the FMA
// two-product.  Every rounding step that must happen exactly as written uses
// the _rn intrinsics, which the compiler never contracts into a fused
// multiply-add: a contraction would change fl(a + b) in a two-sum and break
// its error-free property.
#pragma once

#include "lgf_common.cuh"

namespace lgf {

struct df {
  float h, l;
};

struct cdf {
  df re, im;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a b exactly (FMA two-product)
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// x + y with both parts' errors carried (accurate under cancellation)
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.h, y.h);
  const df t = two_sum(x.l, y.l);
  s.l = __fadd_rn(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return fast_two_sum(s.h, s.l);
}

// x + y, error ~2^-47 (|x| + |y|)
__device__ __forceinline__ df df_add_sloppy(df x, df y) {
  df s = two_sum(x.h, y.h);
  s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
  return fast_two_sum(s.h, s.l);
}

// x + f for an FP32 f
__device__ __forceinline__ df df_add_f(df x, float f) {
  df s = two_sum(x.h, f);
  s.l = __fadd_rn(s.l, x.l);
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.h, -x.l}; }

// x f for an FP32 f
__device__ __forceinline__ df df_mul_f(df x, float f) {
  const df p = two_prod(x.h, f);
  return fast_two_sum(p.h, __fmaf_rn(x.l, f, p.l));
}

// x y, both double-float (the product of the two low parts, ~2^-48 |x y|,
// is dropped)
__device__ __forceinline__ df df_mul(df x, df y) {
  const df p = two_prod(x.h, y.h);
  return fast_two_sum(p.h, __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, p.l)));
}

// ---------------------------------------------------------------------------
// Compensated dot products (the Dot2 scheme of Ogita, Rump and Oishi, 2005):
// the running sum's high part advances by exact two-sums, every product and
// sum error goes into one FP32 low part, and the pair is renormalised once at
// the end.  The result is as accurate as a dot product evaluated in twice the
// working precision, at about 10 operations per term instead of 13 for a
// renormalising double-float addition per term.
// ---------------------------------------------------------------------------
struct dacc {
  float h, l;
};

__device__ __forceinline__ dacc dacc_zero() { return {0.f, 0.f}; }

// a += x y, x and y FP32
__device__ __forceinline__ void dacc_prod(dacc& a, float x, float y) {
  const df p = two_prod(x, y);
  const df s = two_sum(a.h, p.h);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(p.l, s.l));
}

// a += x y, x double-float, y FP32
__device__ __forceinline__ void dacc_prod_df(dacc& a, df x, float y) {
  const df p = two_prod(x.h, y);
  const df s = two_sum(a.h, p.h);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(__fmaf_rn(x.l, y, p.l), s.l));
}

// a += x y, both double-float
__device__ __forceinline__ void dacc_prod_dd(dacc& a, df x, df y) {
  const df p = two_prod(x.h, y.h);
  const df s = two_sum(a.h, p.h);
  a.h = s.h;
  a.l = __fadd_rn(a.l, __fadd_rn(__fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, p.l)), s.l));
}

// a += a first-order (low-part) term x y: it lands in the low part only
__device__ __forceinline__ void dacc_lo(dacc& a, float x, float y) { a.l = __fmaf_rn(x, y, a.l); }

__device__ __forceinline__ df dacc_result(dacc a) { return fast_two_sum(a.h, a.l); }

// 1 / sqrt(n) for a double-float n near 1 (a row norm of a matrix within
// ~1e-3 of unitary): y = rsqrtf(n.h), then with n y^2 = 1 + d, |d| ~ 2^-22,
// 1/sqrt(n) = y (1 - d/2 + 3 d^2 / 8 - ...), whose next term (~2^-68) is far
// below double-float rounding.  d = dh + dl is formed exactly: n.h y^2 - 1 by
// an exact subtraction (Sterbenz), plus the low parts (dl ~ 2^-23, so the
// quadratic term needs the whole d: its cross term 3/4 dh dl is ~2^-45).
__device__ __forceinline__ df df_rsqrt(df n) {
  const float y = rsqrtf(n.h);
  const df t = two_prod(y, y);
  const df m = two_prod(n.h, t.h);
  const float dh = __fsub_rn(m.h, 1.f);
  const float dl = __fmaf_rn(n.h, t.l, __fmaf_rn(n.l, t.h, m.l));
  const float d = __fadd_rn(dh, dl);
  // y (-dh / 2) exactly, the rest to first order
  const df p = two_prod(y, -0.5f * dh);
  const float rest = __fmaf_rn(y, __fmaf_rn(0.375f * d, d, -0.5f * dl), p.l);
  const df q = fast_two_sum(y, p.h);
  return fast_two_sum(q.h, __fadd_rn(q.l, rest));
}

// Exact FP64 value of an FP32 number by bit manipulation (normal numbers and
// zero; FP32 subnormals, below 1.2e-38, map to zero; NaN/Inf to NaN).
__device__ __forceinline__ double fp32_to_fp64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const int e = (int)((u >> 23) & 0xffu);
  if (e == 0) return __longlong_as_double((long long)s);
  if (e == 0xff) return __longlong_as_double(0x7ff8000000000000ll);
  const unsigned long long bits = s | ((unsigned long long)(e - 127 + 1023) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// hi + lo as one FP64 value by one FP64 addition: exact whenever the pair's
// bits span at most 53 binary places, else its FP64 rounding
__device__ __forceinline__ double df_to_double(float h, float l) {
  return fp32_to_fp64_bits(h) + fp32_to_fp64_bits(l);
}

// One link of U' = (1 + eta) U (1 + eta')^dag in double-float, accurate to
// ~2^-48: U and eta = eta(x), eta' = eta(x+mu) in double-float, the first-order
// terms eta U + U eta'^dag by compensated dot products of exact products
// (their hi x lo parts in the low parts), the second-order eta U eta'^dag
// (~1e-10) in FP32.  For the host store and the conversion to FP64 planes.
__device__ __forceinline__ void tail_link_exact(const M3<float>& uh, const cx<float> (&ul)[9], const M3<float>& xh,
                                                const M3<float>& xl, const M3<float>& fh, const M3<float>& fl,
                                                df (&re)[9], df (&im)[9]) {
  M3<float> a, t2;
  mm<float, 3>(a, xh, uh);
  mm_dag<float, 3>(t2, a, fh);  // eta U eta'^dag
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dacc r = {uh.e[i][j].re, ul[i * 3 + j].re}, m = {uh.e[i][j].im, ul[i * 3 + j].im};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // (eta U)_ij += eta_ik U_kj
        const cx<float> x = xh.e[i][k], y = uh.e[k][j], xe = xl.e[i][k], ye = ul[k * 3 + j];
        dacc_prod(r, x.re, y.re);
        dacc_prod(r, -x.im, y.im);
        dacc_prod(m, x.re, y.im);
        dacc_prod(m, x.im, y.re);
        dacc_lo(r, xe.re, y.re);
        dacc_lo(r, -xe.im, y.im);
        dacc_lo(r, x.re, ye.re);
        dacc_lo(r, -x.im, ye.im);
        dacc_lo(m, xe.re, y.im);
        dacc_lo(m, xe.im, y.re);
        dacc_lo(m, x.re, ye.im);
        dacc_lo(m, x.im, ye.re);
        // (U eta'^dag)_ij += U_ik conj(eta'_jk)
        const cx<float> u = uh.e[i][k], f = fh.e[j][k], ue = ul[i * 3 + k], fe = fl.e[j][k];
        dacc_prod(r, u.re, f.re);
        dacc_prod(r, u.im, f.im);
        dacc_prod(m, u.im, f.re);
        dacc_prod(m, -u.re, f.im);
        dacc_lo(r, ue.re, f.re);
        dacc_lo(r, ue.im, f.im);
        dacc_lo(r, u.re, fe.re);
        dacc_lo(r, u.im, fe.im);
        dacc_lo(m, ue.im, f.re);
        dacc_lo(m, -ue.re, f.im);
        dacc_lo(m, u.im, fe.re);
        dacc_lo(m, -u.re, fe.im);
      }
      r.l = __fadd_rn(r.l, t2.e[i][j].re);
      m.l = __fadd_rn(m.l, t2.e[i][j].im);
      re[i * 3 + j] = dacc_result(r);
      im[i * 3 + j] = dacc_result(m);
    }
}

// The tail's gauge step at site s: 1 + eta <- (1 + eps)(1 + eta), eps = X +
// X^2/2, X = h Delta~ from the packed accelerated gradient (c0..c3), eta in
// double-float (eh: hi planes, el: lo planes, 9 complex planes each):
// eta <- eta + X + (X^2/2 + eps eta_hi).  X, exactly anti-Hermitian, enters by
// exact two-sums; only the small Hermitian terms (|X|^2 ~ 1e-10) are rounded
// in FP32.  So 1 + eta stays unitary to O(|X|^3) plus ~1e-17, where rounding
// X + X^2/2 as one FP32 sum would break unitarity by 2^-24 |X| at every step.
__device__ __forceinline__ void tail_eta_site(cx<float> c0, cx<float> c1, cx<float> c2, cx<float> c3, float h,
                                              cx<float>* __restrict__ eh, cx<float>* __restrict__ el, int V, int s) {
  M3<float> X;
  X.e[0][0] = mk<float>(0.f, h * c3.re);
  X.e[1][1] = mk<float>(0.f, h * c3.im);
  X.e[2][2] = mk<float>(0.f, -h * (c3.re + c3.im));
  X.e[0][1] = scale(c0, h);
  X.e[0][2] = scale(c1, h);
  X.e[1][2] = scale(c2, h);
  X.e[1][0] = mk<float>(-h * c0.re, h * c0.im);
  X.e[2][0] = mk<float>(-h * c1.re, h * c1.im);
  X.e[2][1] = mk<float>(-h * c2.re, h * c2.im);
  M3<float> n;
  cx<float> lo[9];  // all of eta's loads issued before any arithmetic
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    n.e[q / 3][q % 3] = eh[q * V + s];
    lo[q] = el[q * V + s];
  }
  // small terms: X^2/2 + (X + X^2/2) eta_hi
  M3<float> Y;
  mm<float, 3>(Y, X, X);
  M3<float> e = X;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Y.e[i][j] = scale(Y.e[i][j], 0.5f);
      e.e[i][j] = e.e[i][j] + Y.e[i][j];
    }
  mm_acc(Y, e, n);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int i = q / 3, j = q % 3;
    df re = two_sum(n.e[i][j].re, X.e[i][j].re);
    df im = two_sum(n.e[i][j].im, X.e[i][j].im);
    re = fast_two_sum(re.h, __fadd_rn(re.l, __fadd_rn(lo[q].re, Y.e[i][j].re)));
    im = fast_two_sum(im.h, __fadd_rn(im.l, __fadd_rn(lo[q].im, Y.e[i][j].im)));
    eh[q * V + s] = mk<float>(re.h, im.h);
    el[q * V + s] = mk<float>(re.l, im.l);
  }
}

}  // namespace lgf
