// In-register FFT of one line of compile-time length L (mixed radix 4, 2, 3,
// 5), used by the per-axis Fourier-acceleration passes.
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
// Twiddles W_L^m = exp(-2 pi i m / L) come from a per-axis table in shared
// memory (all threads read the same entry: broadcast).
#pragma once

#include "lgf_common.cuh"

namespace lgf {
namespace regfft {

constexpr int next_radix(int n) { return n % 4 == 0 ? 4 : (n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : 5)); }

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
constexpr int digit_rev(int L, int p) {
  int k = 0, rem = p, n = L, mult = 1;
  while (n > 1) {
    const int R = next_radix(n);
    n /= R;
    const int d = rem / n;
    rem %= n;
    k += d * mult;
    mult *= R;
  }
  return k;
}

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
    const T h = (T)0.5;
    const T s = (T)0.86602540378443864676;  // sin(2 pi / 3)
    const cx<T> t1 = v[1] + v[2];
    const cx<T> t2 = scale(mul_i(v[1] - v[2], !INV), s);
    const cx<T> m = v[0] - scale(t1, h);
    v[0] = v[0] + t1;
    v[1] = m + t2;
    v[2] = m - t2;
  } else {  // R == 5
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
    const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
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
template <class T, int L, int N>
__device__ __forceinline__ void dif_stages(cx<T>* a, const cx<T>* tw) {
  if constexpr (N > 1) {
    constexpr int R = next_radix(N);
    constexpr int span = N / R;
#pragma unroll
    for (int b = 0; b < L / N; ++b) {
#pragma unroll
      for (int k = 0; k < span; ++k) {
        cx<T> u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = a[b * N + k + r * span];
        dft<T, R, false>(u);
#pragma unroll
        for (int q = 0; q < R; ++q) a[b * N + k + q * span] = (q == 0 || k == 0) ? u[q] : u[q] * tw[q * k * (L / N)];
      }
    }
    dif_stages<T, L, span>(a, tw);
  }
}

// Inverse stages: the innermost forward stage is undone first.
template <class T, int L, int N>
__device__ __forceinline__ void dit_inv_stages(cx<T>* a, const cx<T>* tw) {
  if constexpr (N > 1) {
    constexpr int R = next_radix(N);
    constexpr int span = N / R;
    dit_inv_stages<T, L, span>(a, tw);
#pragma unroll
    for (int b = 0; b < L / N; ++b) {
#pragma unroll
      for (int k = 0; k < span; ++k) {
        cx<T> u[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const cx<T> v = a[b * N + k + q * span];
          u[q] = (q == 0 || k == 0) ? v : mul_cj(v, tw[q * k * (L / N)]);
        }
        dft<T, R, true>(u);
#pragma unroll
        for (int r = 0; r < R; ++r) a[b * N + k + r * span] = u[r];
      }
    }
  }
}

template <class T, int L>
__device__ __forceinline__ void forward(cx<T>* a, const cx<T>* tw) {
  dif_stages<T, L, L>(a, tw);
}

template <class T, int L>
__device__ __forceinline__ void inverse(cx<T>* a, const cx<T>* tw) {
  dit_inv_stages<T, L, L>(a, tw);
}

}  // namespace regfft
}  // namespace lgf
