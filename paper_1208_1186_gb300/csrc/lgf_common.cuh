// Shared device definitions for liblgf: complex arithmetic, SU(3) matrices in
// structure-of-arrays storage, lattice geometry and the state that lets a
// queue of iterations stop on the device once theta is below tolerance.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lgf {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <class T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <class T>
__host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> c;
  c.re = r;
  c.im = i;
  return c;
}
template <class T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <class T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <class T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return mk<T>(a.re, -a.im); }
// a * conj(b)
template <class T>
__device__ __forceinline__ cx<T> mul_cj(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <class T>
__device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk<T>(a.re * s, a.im * s); }
template <class T>
__device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }

template <class D, class S>
__device__ __forceinline__ cx<D> cvt(cx<S> a) { return mk<D>((D)a.re, (D)a.im); }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }

// acc + a*b as four fused multiply-adds
template <class T>
__device__ __forceinline__ cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b) {
  const T re = fmaT(-a.im, b.im, fmaT(a.re, b.re, acc.re));
  const T im = fmaT(a.im, b.re, fmaT(a.re, b.im, acc.im));
  return mk<T>(re, im);
}
// acc + a*conj(b) as four fused multiply-adds
template <class T>
__device__ __forceinline__ cx<T> cmac_cj(cx<T> acc, cx<T> a, cx<T> b) {
  const T re = fmaT(a.im, b.im, fmaT(a.re, b.re, acc.re));
  const T im = fmaT(-a.re, b.im, fmaT(a.im, b.re, acc.im));
  return mk<T>(re, im);
}

// read-only, cached load of one complex element
template <class T>
__device__ __forceinline__ cx<T> ldg(const cx<T>* p);
template <>
__device__ __forceinline__ cx<double> ldg(const cx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<float> ldg(const cx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel
// launched with launch_pdl is set up while its predecessor in the stream
// drains and starts as the predecessor's last CTA exits; it calls pdl_wait()
// before it reads or writes anything (the wait returns once the predecessor
// has completed and its writes are visible).  No kernel here triggers its
// dependents early (griddepcontrol.launch_dependents): dependents scheduled
// before the predecessor's tail held SM resources that tail needed, which
// measured slower than no early trigger at all.  A no-op for a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// hardware reciprocal approximation (PTX rcp.approx.ftz.f32: at most 1 ulp
// from the exact reciprocal, subnormals flushed); used for the Fourier
// acceleration factor, a preconditioner whose last bit does not matter
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// asynchronous global -> shared copy of one complex element (8 or 16 bytes,
// both addresses aligned to the element); complete after cp_async_wait_all
template <class T>
__device__ __forceinline__ void cp_async_elem(cx<T>* sdst, const cx<T>* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(cx<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// 3x3 complex matrices
// ---------------------------------------------------------------------------
template <class T>
struct M3 {
  cx<T> e[3][3];
};

// row 3 of an SU(3) matrix from rows 1 and 2: conj(r1 x r2)
template <class T>
__device__ __forceinline__ void complete_row3(M3<T>& m) {
  m.e[2][0] = conj(m.e[0][1] * m.e[1][2] - m.e[0][2] * m.e[1][1]);
  m.e[2][1] = conj(m.e[0][2] * m.e[1][0] - m.e[0][0] * m.e[1][2]);
  m.e[2][2] = conj(m.e[0][0] * m.e[1][1] - m.e[0][1] * m.e[1][0]);
}

// Load a matrix stored as NC complex planes of V elements each (NC = 9: all
// entries row-major; NC = 6: rows 1-2, row 3 rebuilt).
template <class T, int NC>
__device__ __forceinline__ M3<T> load_m3(const cx<T>* __restrict__ base, int64_t V, int64_t s) {
  M3<T> m;
#pragma unroll
  for (int c = 0; c < NC; ++c) m.e[c / 3][c % 3] = ldg(base + c * V + s);
  if (NC == 6) complete_row3(m);
  return m;
}

// The same with 32-bit element offsets (valid while NC * 4 * V < 2^31, which
// the 64-site extent limit guarantees: at most 36 * 64^4 elements).
template <class T, int NC>
__device__ __forceinline__ M3<T> load_m3i(const cx<T>* __restrict__ base, int V, int s) {
  M3<T> m;
#pragma unroll
  for (int c = 0; c < NC; ++c) m.e[c / 3][c % 3] = ldg(base + (c * V + s));
  if (NC == 6) complete_row3(m);
  return m;
}

__device__ __forceinline__ void site_coords_i(const int L[4], int s, int c[4]) {
  c[0] = s % L[0];
  s /= L[0];
  c[1] = s % L[1];
  s /= L[1];
  c[2] = s % L[2];
  c[3] = s / L[2];
}

template <class T, int NC>
__device__ __forceinline__ void store_m3(cx<T>* __restrict__ base, int64_t V, int64_t s, const M3<T>& m) {
#pragma unroll
  for (int c = 0; c < NC; ++c) base[c * V + s] = m.e[c / 3][c % 3];
}

// c = a * b for the first ROWS rows of c
template <class T, int ROWS = 3>
__device__ __forceinline__ void mm(M3<T>& c, const M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < ROWS; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = a.e[i][0] * b.e[0][j];
      acc = cmac(acc, a.e[i][1], b.e[1][j]);
      c.e[i][j] = cmac(acc, a.e[i][2], b.e[2][j]);
    }
}

// c = a * b^dagger for the first ROWS rows of c
template <class T, int ROWS = 3>
__device__ __forceinline__ void mm_dag(M3<T>& c, const M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < ROWS; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = mul_cj(a.e[i][0], b.e[j][0]);
      acc = cmac_cj(acc, a.e[i][1], b.e[j][1]);
      c.e[i][j] = cmac_cj(acc, a.e[i][2], b.e[j][2]);
    }
}

// c += a * b
template <class T>
__device__ __forceinline__ void mm_acc(M3<T>& c, const M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = cmac(c.e[i][j], a.e[i][0], b.e[0][j]);
      acc = cmac(acc, a.e[i][1], b.e[1][j]);
      c.e[i][j] = cmac(acc, a.e[i][2], b.e[2][j]);
    }
}

// c += a * b^dagger
template <class T>
__device__ __forceinline__ void mm_dag_acc(M3<T>& c, const M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = cmac_cj(c.e[i][j], a.e[i][0], b.e[j][0]);
      acc = cmac_cj(acc, a.e[i][1], b.e[j][1]);
      c.e[i][j] = cmac_cj(acc, a.e[i][2], b.e[j][2]);
    }
}

// Project onto SU(3): Gram-Schmidt on rows 1 and 2, row 3 = conj(r1 x r2).
template <class T>
__device__ __forceinline__ void reunitarize(M3<T>& m) {
  T n1 = norm2(m.e[0][0]) + norm2(m.e[0][1]) + norm2(m.e[0][2]);
  T inv1 = rsqrt(n1);
#pragma unroll
  for (int j = 0; j < 3; ++j) m.e[0][j] = scale(m.e[0][j], inv1);
  // <r1, r2> = sum conj(r1_j) r2_j
  cx<T> ip = mul_cj(m.e[1][0], m.e[0][0]);
  ip = ip + mul_cj(m.e[1][1], m.e[0][1]);
  ip = ip + mul_cj(m.e[1][2], m.e[0][2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) m.e[1][j] = m.e[1][j] - ip * m.e[0][j];
  T n2 = norm2(m.e[1][0]) + norm2(m.e[1][1]) + norm2(m.e[1][2]);
  T inv2 = rsqrt(n2);
#pragma unroll
  for (int j = 0; j < 3; ++j) m.e[1][j] = scale(m.e[1][j], inv2);
  complete_row3(m);
}

// exp(X) of a 3x3 complex matrix of moderate norm (here traceless
// anti-Hermitian, |X| < ~2) by scaling and squaring with a Taylor polynomial
// (Moler and Van Loan, "Nineteen dubious ways to compute the exponential of a
// matrix", 2003, the Taylor method with scaling and squaring): Y = X / 2^q
// with squared Frobenius norm <= 1/4, exp(Y) by Horner's rule on its Taylor
// series to degree 16 (FP64; remainder below 0.5^17 / 17! ~ 2e-20) or 9
// (FP32; ~6e-9), then q squarings.  At most 30 halvings, so a non-finite
// input ends in a non-finite result instead of a long loop.
template <class T>
__device__ __forceinline__ M3<T> expm_taylor(const M3<T>& X) {
  T n2 = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) n2 += norm2(X.e[i][j]);
  int q = 0;
  T sc = 1;
  while (n2 > (T)0.25 && q < 30) {
    n2 *= (T)0.25;
    sc *= (T)0.5;
    ++q;
  }
  M3<T> Y, E;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Y.e[i][j] = scale(X.e[i][j], sc);
      E.e[i][j] = mk<T>(i == j ? (T)1 : (T)0, 0);
    }
  constexpr int kDeg = sizeof(T) == 8 ? 16 : 9;
#pragma unroll 1
  for (int k = kDeg; k >= 1; --k) {  // E <- 1 + Y E / k
    M3<T> t;
    mm<T, 3>(t, Y, E);
    const T inv = (T)1 / (T)k;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        E.e[i][j] = scale(t.e[i][j], inv);
        if (i == j) E.e[i][j].re += (T)1;
      }
  }
#pragma unroll 1
  for (int r = 0; r < q; ++r) {
    M3<T> t;
    mm<T, 3>(t, E, E);
    E = t;
  }
  return E;
}

// The whole traceless anti-Hermitian h Delta~ from its packed form c0..c3
// (Delta~_01, Delta~_02, Delta~_12, Im Delta~_00 + i Im Delta~_11).
template <class T>
__device__ __forceinline__ M3<T> unpack_ah(cx<T> c0, cx<T> c1, cx<T> c2, cx<T> c3, T h) {
  M3<T> X;
  X.e[0][0] = mk<T>(0, h * c3.re);
  X.e[1][1] = mk<T>(0, h * c3.im);
  X.e[2][2] = mk<T>(0, -h * (c3.re + c3.im));
  X.e[0][1] = scale(c0, h);
  X.e[0][2] = scale(c1, h);
  X.e[1][2] = scale(c2, h);
  X.e[1][0] = mk<T>(-h * c0.re, h * c0.im);
  X.e[2][0] = mk<T>(-h * c1.re, h * c1.im);
  X.e[2][1] = mk<T>(-h * c2.re, h * c2.im);
  return X;
}

// ---------------------------------------------------------------------------
// lattice geometry, passed by value to every kernel
// ---------------------------------------------------------------------------
struct Geom {
  int L[4];         // Lx, Ly, Lz, Lt
  int64_t stride[4];  // 1, Lx, Lx*Ly, Lx*Ly*Lz
  int64_t V;
  // ceil(2^32 / L) for L = Lx, Ly, Lz (geom_init_rcp): the quotient s / L is
  // __umulhi(s, rcp) exactly for 0 <= s < 2^32 / L, i.e. for every site index
  // of a lattice with extents <= 64 (V <= 2^24 < 2^26)
  unsigned rcp[3];
};

inline void geom_init_rcp(Geom& g) {
  for (int a = 0; a < 3; ++a) g.rcp[a] = 0xFFFFFFFFu / (unsigned)g.L[a] + 1u;
}

// coordinates of site s by multiply-high reciprocals (three integer
// multiplies instead of three divisions); needs geom_init_rcp
__device__ __forceinline__ void site_coords_r(const Geom& g, int s, int c[4]) {
  const unsigned u = (unsigned)s;
  const unsigned q0 = __umulhi(u, g.rcp[0]);
  const unsigned q1 = __umulhi(q0, g.rcp[1]);
  const unsigned q2 = __umulhi(q1, g.rcp[2]);
  c[0] = (int)(u - q0 * (unsigned)g.L[0]);
  c[1] = (int)(q0 - q1 * (unsigned)g.L[1]);
  c[2] = (int)(q1 - q2 * (unsigned)g.L[2]);
  c[3] = (int)q2;
}

__device__ __forceinline__ void site_coords(const Geom& g, int64_t s, int c[4]) {
  int64_t r = s;
  c[0] = (int)(r % g.L[0]);
  r /= g.L[0];
  c[1] = (int)(r % g.L[1]);
  r /= g.L[1];
  c[2] = (int)(r % g.L[2]);
  c[3] = (int)(r / g.L[2]);
}

// site index of x - mu (periodic)
__device__ __forceinline__ int64_t site_back(const Geom& g, int64_t s, const int c[4], int mu) {
  return c[mu] > 0 ? s - g.stride[mu] : s + (int64_t)(g.L[mu] - 1) * g.stride[mu];
}
// site index of x + mu (periodic)
__device__ __forceinline__ int64_t site_fwd(const Geom& g, int64_t s, const int c[4], int mu) {
  return c[mu] < g.L[mu] - 1 ? s + g.stride[mu] : s - (int64_t)(g.L[mu] - 1) * g.stride[mu];
}

// ---------------------------------------------------------------------------
// device-side iteration state
// ---------------------------------------------------------------------------
// The final reduction of every iteration writes F and theta here and decides
// whether the update of that iteration goes ahead.  Every later kernel of the
// queue reads `done` first and returns at once when it is set, so a host can
// queue many iterations and still stop exactly at the first theta < tol.
struct DevState {
  double F;          // F of the links before the latest update
  double theta;      // theta of the same links
  int done;          // 1: no further update is applied
  int iters;         // updates applied since the last reset
  int nonfinite;     // F or theta was NaN/Inf
  int max_iter;      // stop once iters reaches this (fix mode)
  double tol;        // stop once theta < tol (fix mode; < 0 disables)
  int hist_cap;
  unsigned int arrive;  // blocks of the current gradient launch that are done
  double* hist;      // theta before update n, n < hist_cap
  int stall;         // also stop once theta < 1e-6 has not halved within 8 updates
  int stall_iters;   // update count at the reference theta
  double stall_ref;  // reference theta of the stall rule (0: none yet)
  int use_cond;      // the queue is a device-side graph loop: set its condition
  unsigned long long cond;  // the loop's cudaGraphConditionalHandle
};

}  // namespace lgf
