// In-register FFT of one line of compile-time length L (mixed radix 4, 2, 3,
// 5), used by the per-axis Fourier-acceleration passes.
//
// Radix order RO: 0 takes the radices greedily (4 while 4 divides what is
// left, then 2, 3, 5: 32 = 4 4 2, 48 = 4 4 3); 1 takes the same factors in
// the reverse order (32 = 2 4 4, 48 = 3 4 4).  Both are exact transforms of
// the same line; they differ in which twiddles multiply which stage, hence in
// instruction count and FP32 rounding, and the autotuner chooses between them
// per extent.  The digit-reversed output order depends on RO.
//
// Forward: decimation in frequency (Sande-Tukey), in place, natural-order
// input, output in mixed-radix digit-reversed order: after dif<L>, element p
// holds frequency digit_rev(L, p).  Inverse: decimation in time, the exact
// reverse of the forward stages (conjugate twiddles, conjugate butterflies),
// taking digit-reversed input and giving natural-order output, unnormalised.
// A forward pass followed by the inverse pass therefore never needs a
// permutation; the acceleration factor is applied at digit-reversed indices.
//
// With L a template constant every loop unrolls and every index, radix and
// twiddle index is a compile-time constant: the line stays in registers.
// Twiddles W_L^m = exp(-2 pi i m / L) are compile-time constants (every
// stage index is a template constant), so they become instruction immediates
// or constant-bank operands: no table, no shared-memory loads, no registers.
// Multiples of a quarter turn are exact sign/swap operations.
#pragma once

#include <type_traits>

#include "lgf_common.cuh"

namespace lgf {
namespace regfft {

constexpr int next_radix(int n) { return n % 4 == 0 ? 4 : (n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : 5)); }

// the last radix of n's order-0 factorisation
constexpr int last_radix0(int n) {
  int r = 1;
  while (n > 1) {
    r = next_radix(n);
    n /= r;
  }
  return r;
}

// radix of the stage that splits a sub-transform of length n, in order RO
constexpr int stage_radix(int n, int ro) { return ro == 0 ? next_radix(n) : last_radix0(n); }

// true if the two radix orders give different stage sequences for length L
constexpr bool orders_differ(int L) {
  int a = L, b = L;
  while (a > 1 && b > 1) {
    const int ra = stage_radix(a, 0), rb = stage_radix(b, 1);
    if (ra != rb) return true;
    a /= ra;
    b /= rb;
  }
  return false;
}

constexpr bool supported(int n) {
  if (n < 2) return false;
  while (n > 1) {
    const int r = next_radix(n);
    if (n % r != 0) return false;
    n /= r;
  }
  return true;
}

// frequency index held at position p after the forward transform
constexpr int digit_rev(int L, int p, int ro = 0) {
  int k = 0, rem = p, n = L, mult = 1;
  while (n > 1) {
    const int R = stage_radix(n, ro);
    n /= R;
    const int d = rem / n;
    rem %= n;
    k += d * mult;
    mult *= R;
  }
  return k;
}

// ---------------------------------------------------------------------------
// cos and sin of 2 pi m / L at compile time.  The angle is reduced to the first
// octant with exact integer arithmetic (8 m = o L + rem), then a Taylor series
// on [0, pi/4] (terms beyond x^25 / 25! are below 1e-27) gives the value to a
// few units in the last place of double; octant symmetries give exact zeros,
// ones and mirrored values.
// ---------------------------------------------------------------------------
constexpr double kTwoPiOver8 = 0.78539816339744830961566084581987572;  // pi / 4

constexpr double poly_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n <= 12; ++n) {
    term *= -x * x / (double)((2 * n) * (2 * n + 1));
    sum += term;
  }
  return sum;
}

constexpr double poly_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n <= 12; ++n) {
    term *= -x * x / (double)((2 * n - 1) * (2 * n));
    sum += term;
  }
  return sum;
}

// {cos, sin} of 2 pi m / L; which = 0 for cos, 1 for sin
constexpr double turn_cs(int m, int L, int which) {
  m = ((m % L) + L) % L;
  const int e = 8 * m, o = e / L, rem = e - o * L;
  const double phi = kTwoPiOver8 * (double)rem / (double)L;        // o pi/4 + phi
  const double psi = kTwoPiOver8 * (double)(L - rem) / (double)L;  // (o+1) pi/4 - psi
  const bool zero = rem == 0;
  const double cp = zero ? 1.0 : poly_cos(phi), sp = zero ? 0.0 : poly_sin(phi);
  const double cq = poly_cos(psi), sq = poly_sin(psi);
  double c = 0.0, s = 0.0;
  switch (o) {
    case 0: c = cp; s = sp; break;
    case 1: c = sq; s = cq; break;
    case 2: c = -sp; s = cp; break;
    case 3: c = -cq; s = sq; break;
    case 4: c = -cp; s = -sp; break;
    case 5: c = -sq; s = -cq; break;
    case 6: c = sp; s = -cp; break;
    default: c = cq; s = -sq; break;
  }
  return which == 0 ? c : s;
}

template <int L, int M>
struct Twiddle {  // W_L^M = exp(-2 pi i M / L)
  static constexpr int m = ((M % L) + L) % L;
  static constexpr bool quarter = (4 * m) % L == 0;  // W in {1, -i, -1, i}
  static constexpr int q = quarter ? 4 * m / L : -1;
  static constexpr double re = turn_cs(m, L, 0);
  static constexpr double im = -turn_cs(m, L, 1);
};

// v * W_L^M (CONJ: v * conj(W_L^M))
template <class T, int L, int M, bool CONJ>
__device__ __forceinline__ cx<T> mul_tw(cx<T> v) {
  using W = Twiddle<L, M>;
  if constexpr (W::quarter) {
    constexpr int q = CONJ ? (4 - W::q) % 4 : W::q;  // W = (-i)^q
    if constexpr (q == 0) return v;
    else if constexpr (q == 1) return mk<T>(v.im, -v.re);
    else if constexpr (q == 2) return mk<T>(-v.re, -v.im);
    else return mk<T>(-v.im, v.re);
  } else {
    constexpr T wr = (T)W::re;
    constexpr T wi = CONJ ? (T)-W::im : (T)W::im;
    return mk<T>(fmaT(v.re, wr, -v.im * wi), fmaT(v.re, wi, v.im * wr));
  }
}

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// 4 sin^2(pi k / L) (the lattice momentum squared of one axis), for the
// frequency k held at position P after the forward transform of order RO
template <int L, int P, int RO = 0>
struct MomentumSq {
  static constexpr double s = turn_cs(digit_rev(L, P, RO), 2 * L, 1);  // sin(2 pi k / (2 L))
  static constexpr double value = 4.0 * s * s;
};

template <class T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a, bool neg) {  // neg ? -i*a : +i*a
  return neg ? mk<T>(a.im, -a.re) : mk<T>(-a.im, a.re);
}

// R-point DFT in place; forward e^{-2 pi i/R}, inverse e^{+2 pi i/R}
template <class T, int R, bool INV>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 2) {
    const cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 4) {
    const cx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
    const cx<T> s13 = v[1] + v[3], d13 = mul_i(v[1] - v[3], !INV);
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = d02 + d13;
    v[3] = d02 - d13;
  } else if constexpr (R == 3) {
    constexpr T h = (T)0.5;
    constexpr T s = (T)turn_cs(1, 3, 1);  // sin(2 pi / 3)
    const cx<T> t1 = v[1] + v[2];
    const cx<T> t2 = scale(mul_i(v[1] - v[2], !INV), s);
    const cx<T> m = v[0] - scale(t1, h);
    v[0] = v[0] + t1;
    v[1] = m + t2;
    v[2] = m - t2;
  } else {  // R == 5
    constexpr T c1 = (T)turn_cs(1, 5, 0), c2 = (T)turn_cs(2, 5, 0);  // cos(2 pi / 5), cos(4 pi / 5)
    constexpr T s1 = (T)turn_cs(1, 5, 1), s2 = (T)turn_cs(2, 5, 1);  // sin(2 pi / 5), sin(4 pi / 5)
    const cx<T> a1 = v[1] + v[4], b1 = v[1] - v[4];
    const cx<T> a2 = v[2] + v[3], b2 = v[2] - v[3];
    const cx<T> p1 = v[0] + scale(a1, c1) + scale(a2, c2);
    const cx<T> p2 = v[0] + scale(a1, c2) + scale(a2, c1);
    const cx<T> q1 = mul_i(scale(b1, s1) + scale(b2, s2), !INV);
    const cx<T> q2 = mul_i(scale(b1, s2) - scale(b2, s1), !INV);
    v[0] = v[0] + a1 + a2;
    v[1] = p1 + q1;
    v[4] = p1 - q1;
    v[2] = p2 + q2;
    v[3] = p2 - q2;
  }
}

// Forward stages on sub-transforms of length N (called with N = L).
template <class T, int L, int N, int RO>
__device__ __forceinline__ void dif_stages(cx<T>* a) {
  if constexpr (N > 1) {
    constexpr int R = stage_radix(N, RO);
    constexpr int span = N / R;
#pragma unroll
    for (int b = 0; b < L / N; ++b) {
      static_for<0, span>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        cx<T> u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = a[b * N + k + r * span];
        dft<T, R, false>(u);
        a[b * N + k] = u[0];
        static_for<1, R>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          a[b * N + k + q * span] = mul_tw<T, L, q * k * (L / N), false>(u[q]);
        });
      });
    }
    dif_stages<T, L, span, RO>(a);
  }
}

// Inverse stages: the innermost forward stage is undone first.
template <class T, int L, int N, int RO>
__device__ __forceinline__ void dit_inv_stages(cx<T>* a) {
  if constexpr (N > 1) {
    constexpr int R = stage_radix(N, RO);
    constexpr int span = N / R;
    dit_inv_stages<T, L, span, RO>(a);
#pragma unroll
    for (int b = 0; b < L / N; ++b) {
      static_for<0, span>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        cx<T> u[R];
        u[0] = a[b * N + k];
        static_for<1, R>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          u[q] = mul_tw<T, L, q * k * (L / N), true>(a[b * N + k + q * span]);
        });
        dft<T, R, true>(u);
#pragma unroll
        for (int r = 0; r < R; ++r) a[b * N + k + r * span] = u[r];
      });
    }
  }
}

template <class T, int L, int RO = 0>
__device__ __forceinline__ void forward(cx<T>* a) {
  dif_stages<T, L, L, RO>(a);
}

template <class T, int L, int RO = 0>
__device__ __forceinline__ void inverse(cx<T>* a) {
  dit_inv_stages<T, L, L, RO>(a);
}

// ---------------------------------------------------------------------------
// Pair-split transforms ("radix order 2"): a line of even length L shared by
// two lanes l and l ^ 1 of a warp, half h = l & 1 holding elements
// h L/2 ... h L/2 + L/2 - 1 in natural order.  The forward transform's first
// stage is the radix-2 decimation-in-frequency butterfly between the halves,
// done across the pair with shuffles; each lane then transforms its half
// (length L/2, greedy radix order 0) in registers.  Afterwards element p of
// half h holds frequency 2 digit_rev(L/2, p) + h.  The inverse undoes the
// stages in reverse order and returns the halves in natural order.  For L = 8
// and L = 32 the stage sequence (2, then 4s) is that of radix order 1, and
// the results are bit-identical to it.  Both lanes of every pair must call
// these (full-warp shuffles).

constexpr int pair_freq(int L, int p, int h) { return 2 * digit_rev(L / 2, p, 0) + h; }

constexpr bool pair_supported(int L) { return L % 2 == 0 && L >= 4 && supported(L / 2); }

template <int L, int P, int HALF>
struct MomentumSqPair {
  static constexpr double s = turn_cs(pair_freq(L, P, HALF), 2 * L, 1);  // sin(pi k / L)
  static constexpr double value = 4.0 * s * s;
};

template <class T>
__device__ __forceinline__ cx<T> shfl_pair(cx<T> v) {
  return mk<T>(__shfl_xor_sync(0xffffffffu, v.re, 1), __shfl_xor_sync(0xffffffffu, v.im, 1));
}

template <class T, int L>
__device__ __forceinline__ void forward_pair(cx<T>* a, int h) {
  constexpr int H = L / 2;
  static_for<0, H>([&](auto nc) {
    constexpr int n = decltype(nc)::value;
    const cx<T> o = shfl_pair(a[n]);
    // half 0: a_n + a_{n+H}; half 1: (a_n - a_{n+H}) W_L^n
    const cx<T> sum = a[n] + o;
    const cx<T> dif = mul_tw<T, L, n, false>(o - a[n]);
    a[n] = h ? dif : sum;
  });
  dif_stages<T, H, H, 0>(a);
}

template <class T, int L>
__device__ __forceinline__ void inverse_pair(cx<T>* a, int h) {
  constexpr int H = L / 2;
  dit_inv_stages<T, H, H, 0>(a);
  static_for<0, H>([&](auto nc) {
    constexpr int n = decltype(nc)::value;
    // half 1 sends b_n conj(W_L^n); half 0 sends a_n
    const cx<T> mine = h ? mul_tw<T, L, n, true>(a[n]) : a[n];
    const cx<T> o = shfl_pair(mine);
    a[n] = h ? o - mine : mine + o;
  });
}

}  // namespace regfft
}  // namespace lgf
