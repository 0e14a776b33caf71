// FP64 tail by defect correction.
//
// Near convergence (theta < 1e-8 when the tail starts) the gauge step
// g = reunit(1 + X), X = alpha/2 Delta~, differs from the identity by
// |X| < 1e-5.  The links must be FP64 to resolve a gradient of that size
// (Delta is a difference of O(1) link entries), but the step itself only
// needs FP32 *relative* precision.  So the tail keeps FP64 links and:
//
//   k_gradient_tail  Delta and F/theta from the FP64 links, in FP64
//                    (additions only), Delta stored as FP32 for the FFT;
//   (FP32 Fourier acceleration of the packed gradient)
//   k_tail_step      eps = X + X^2/2 in FP32 (g = 1 + eps is the exponential
//                    to second order: unitary to O(|X|^3), below FP64
//                    rounding; it agrees with reunit(1 + X) to O(|X|^2));
//   k_tail_update    U += eps U + U eps(x+mu)^dag + eps U eps(x+mu)^dag, the
//                    correction in FP32 (from FP32-rounded U; its error is
//                    |eps| * 2^-24 ~ 1e-13 |eps|), accumulated in FP64.
//
// FP64 work per site drops from ~2.5k operations (FP64 products, FFT,
// Gram-Schmidt) to ~0.3k (sums).  Even those sums bound the kernels on this
// GPU, whose FP64 pipe runs at 1/62 of FP32.  So by default the tail keeps its
// links in double-float form instead: two FP32 planes per entry, value =
// hi + lo with |lo| <= ulp(hi)/2 (48 significant bits, relative rounding
// about 2^-47), and does every operation on the FP32 pipe with error-free
// transformations (Knuth's two-sum, Dekker's fast-two-sum, the FMA
// two-product):
//
//   k_tail_start_df     U = g U_loaded g(x+mu)^dag from the FP64 input and the
//                       FP64-reunitarised gauge, both split exactly into
//                       hi + lo by bit manipulation, products in double-float;
//   k_gradient_tail_df  Delta by double-float sums, F summed in double-float
//                       per warp, D stored as FP32;
//   k_tail_update_df    U += the FP32 correction, a double-float addition;
//   k_df_to_fp64        the final links back to FP64 (exact conversions, one
//                       FP64 addition per real).
//
// The tail's own error budget (each FP32 correction is exact to |eps| 2^-24,
// about 1e-12 at the first step) is far above the double-float rounding.
#include "lgf_kernels.cuh"
#include "lgf_reduce.cuh"

namespace lgf {

namespace {

__global__ void __launch_bounds__(256) k_gradient_tail(const cx<double>* __restrict__ U, cx<float>* __restrict__ D,
                                                       double2* __restrict__ partial, const Geom geo, DevState* st,
                                                       int mode, double normF, double normT) {
  pdl_wait();
  if (queue_stopped(st, mode)) return;
  const int V = (int)geo.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double fsum = 0.0, tsum = 0.0;
  if (s < V) {
    int c[4];
    site_coords_i(geo.L, s, c);
    M3<double> A;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A.e[i][j] = mk<double>(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const cx<double>* base = U + mu * 9 * V;
      const int st_mu = (int)geo.stride[mu];
      const int sb = c[mu] > 0 ? s - st_mu : s + (geo.L[mu] - 1) * st_mu;
      const M3<double> own = load_m3i<double, 9>(base, V, s);
      const M3<double> back = load_m3i<double, 9>(base, V, sb);
      fsum += own.e[0][0].re + own.e[1][1].re + own.e[2][2].re;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A.e[i][j] = A.e[i][j] + (back.e[i][j] - own.e[i][j]);
    }
    const cx<double> d01 = A.e[0][1] - conj(A.e[1][0]);
    const cx<double> d02 = A.e[0][2] - conj(A.e[2][0]);
    const cx<double> d12 = A.e[1][2] - conj(A.e[2][1]);
    const double a0 = 2 * A.e[0][0].im, a1 = 2 * A.e[1][1].im, a2 = 2 * A.e[2][2].im;
    const double tr = (a0 + a1 + a2) / 3.0;
    const double i0 = a0 - tr, i1 = a1 - tr, i2 = -(i0 + i1);
    D[s] = cvt<float>(d01);
    D[V + s] = cvt<float>(d02);
    D[2 * V + s] = cvt<float>(d12);
    D[3 * V + s] = mk<float>((float)i0, (float)i1);
    tsum = 2 * (norm2(d01) + norm2(d02) + norm2(d12)) + i0 * i0 + i1 * i1 + i2 * i2;
  }
  grid_reduce<double>(fsum, tsum, partial, st, normF, normT, mode);
}

// eps = X + X^2 / 2, X = h Delta~ (traceless anti-Hermitian), 9 FP32 planes
__global__ void __launch_bounds__(256) k_tail_step(const cx<float>* __restrict__ D, cx<float>* __restrict__ eps,
                                                   int V, float h, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const cx<float> c0 = ldg(D + s), c1 = ldg(D + V + s), c2 = ldg(D + 2 * V + s), c3 = ldg(D + 3 * V + s);
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
  M3<float> X2;
  mm<float, 3>(X2, X, X);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int i = q / 3, j = q % 3;
    eps[q * V + s] = X.e[i][j] + scale(X2.e[i][j], 0.5f);
  }
}

// U_mu(x) += eps(x) U + U eps(x+mu)^dag + eps(x) U eps(x+mu)^dag
__global__ void __launch_bounds__(256) k_tail_update(cx<double>* U, const cx<float>* __restrict__ eps, const Geom geo,
                                                     const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int V = (int)geo.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords_i(geo.L, s, c);
  const M3<float> ex = load_m3i<float, 9>(eps, V, s);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    cx<double>* base = U + mu * 9 * V;
    const int st_mu = (int)geo.stride[mu];
    const int sf = c[mu] < geo.L[mu] - 1 ? s + st_mu : s - (geo.L[mu] - 1) * st_mu;
    const M3<float> ef = load_m3i<float, 9>(eps, V, sf);
    M3<double> u;
    M3<float> uf;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      u.e[q / 3][q % 3] = base[q * V + s];
      uf.e[q / 3][q % 3] = cvt<float>(u.e[q / 3][q % 3]);
    }
    M3<float> a, d;
    mm<float, 3>(a, ex, uf);       // eps U
    mm_dag<float, 3>(d, uf, ef);   // U eps'^dag
    mm_dag_acc(d, a, ef);          // + eps U eps'^dag
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int i = q / 3, j = q % 3;
      const cx<float> delta = a.e[i][j] + d.e[i][j];
      base[q * V + s] = u.e[i][j] + cvt<double>(delta);
    }
  }
}

// ---------------------------------------------------------------------------
// double-float arithmetic (FP32 pairs)
// ---------------------------------------------------------------------------
struct df {
  float h, l;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

// x + y with both parts' errors carried (accurate under cancellation)
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.h, y.h);
  const df t = two_sum(x.l, y.l);
  s.l += t.h;
  s = fast_two_sum(s.h, s.l);
  s.l += t.l;
  return fast_two_sum(s.h, s.l);
}

// x + f for an FP32 f
__device__ __forceinline__ df df_add_f(df x, float f) {
  df s = two_sum(x.h, f);
  s.l += x.l;
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.h, -x.l}; }

struct cdf {
  df re, im;
};

// Exact split of an FP64 value into hi + lo by bit manipulation (no FP64
// arithmetic): hi = x truncated to 24 significant bits, lo = the remaining
// (up to 29) bits rounded to 24.  |x| < 2^-100 (no SU(3) entry that matters)
// maps to 0; NaN/Inf map to NaN so that they surface in F and theta.
__device__ __forceinline__ df split_fp64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffull);
  if (e == 0x7ff) return {__int_as_float(0x7fc00000), 0.f};
  const int E = e - 1023;
  if (e == 0 || E < -100) return {0.f, 0.f};
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29));
  const int se = E - 52 + 127;  // lo = r 2^(E-52)
  const float scale = se >= 1 ? __uint_as_float((unsigned)se << 23) : 0.f;
  const float lo = __uint2float_rn((unsigned)(m & 0x1fffffffull)) * scale;
  return {hi, sign ? -lo : lo};
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

__device__ __forceinline__ cdf load_cdf(const cx<float>* __restrict__ h, const cx<float>* __restrict__ l, int i) {
  const cx<float> a = ldg(h + i), b = ldg(l + i);
  return {{a.re, b.re}, {a.im, b.im}};
}

// U_mu(x) = g(x) U_loaded,mu(x) g(x+mu)^dag, one thread per (site, mu), from
// the exact splits g = Gh + Gl and U = Uh + Ul of the FP64 values:
//   Gh Uh Gh'^dag in double-float (Gh Uh from exact FMA products of FP32
//   numbers, then double-float times FP32), plus the first-order terms
//   (Gl Uh + Gh Ul) Gh'^dag + (Gh Uh) Gl'^dag in FP32 (they are ~2^-24 of the
//   result, so FP32 rounding leaves ~2^-48); the second-order terms (~2^-48)
//   are dropped.
__device__ __forceinline__ df df_add_sloppy(df x, df y) {  // error ~2^-47 (|x| + |y|)
  df s = two_sum(x.h, y.h);
  s.l += x.l + y.l;
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df df_mul_f(df x, float f) {
  const float p = x.h * f;
  float e = fmaf(x.h, f, -p);
  e = fmaf(x.l, f, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ void split_matrix(const cx<double>* __restrict__ p, int V, int s, cx<float> (&h)[9],
                                             cx<float> (&l)[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const cx<double> v = ldg(p + q * V + s);
    const df re = split_fp64(v.re), im = split_fp64(v.im);
    h[q] = mk<float>(re.h, im.h);
    l[q] = mk<float>(re.l, im.l);
  }
}

// one thread per (site, mu)
__global__ void __launch_bounds__(128) k_tail_start_df(const cx<double>* __restrict__ Uin,
                                                       const cx<double>* __restrict__ g, cx<float>* __restrict__ Uh,
                                                       cx<float>* __restrict__ Ul, const Geom geo) {
  const int V = (int)geo.V;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * V) return;
  const int s = i % V, mu = i / V;  // consecutive threads: consecutive sites of one direction
  int c[4];
  site_coords_i(geo.L, s, c);
  const int st_mu = (int)geo.stride[mu];
  const int sf = c[mu] < geo.L[mu] - 1 ? s + st_mu : s - (geo.L[mu] - 1) * st_mu;
  cx<float> Gh[9], Gl[9], UH[9], UL[9];
  split_matrix(g, V, s, Gh, Gl);
  split_matrix(Uin + mu * 9 * V, V, s, UH, UL);
  cdf W[9];        // Gh Uh, double-float
  cx<float> P[9];  // Gl Uh + Gh Ul, FP32
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      df re = {0.f, 0.f}, im = {0.f, 0.f};
      cx<float> p = mk<float>(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cx<float> x = Gh[a * 3 + k], y = UH[k * 3 + b];
        re = df_add_sloppy(re, two_prod(x.re, y.re));
        re = df_add_sloppy(re, df_neg(two_prod(x.im, y.im)));
        im = df_add_sloppy(im, two_prod(x.re, y.im));
        im = df_add_sloppy(im, two_prod(x.im, y.re));
        p = cmac(p, Gl[a * 3 + k], y);
        p = cmac(p, x, UL[k * 3 + b]);
      }
      W[a * 3 + b] = {re, im};
      P[a * 3 + b] = p;
    }
  cx<float> Fh[9], Fl[9];
  split_matrix(g, V, sf, Fh, Fl);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      df re = {0.f, 0.f}, im = {0.f, 0.f};
      cx<float> corr = mk<float>(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // W conj(Fh): re += W.re Fh.re + W.im Fh.im, im += W.im Fh.re - W.re Fh.im
        const cdf w = W[a * 3 + k];
        const cx<float> f = Fh[b * 3 + k];
        re = df_add_sloppy(re, df_mul_f(w.re, f.re));
        re = df_add_sloppy(re, df_mul_f(w.im, f.im));
        im = df_add_sloppy(im, df_mul_f(w.im, f.re));
        im = df_add_sloppy(im, df_neg(df_mul_f(w.re, f.im)));
        corr = cmac_cj(corr, P[a * 3 + k], f);
        corr = cmac_cj(corr, mk<float>(w.re.h, w.im.h), Fl[b * 3 + k]);
      }
      re = df_add_f(re, corr.re);
      im = df_add_f(im, corr.im);
      const int o = (mu * 9 + a * 3 + b) * V + s;
      Uh[o] = mk<float>(re.h, im.h);
      Ul[o] = mk<float>(re.l, im.l);
    }
}

// Delta and F/theta from double-float links; D stored as FP32
__global__ void __launch_bounds__(256) k_gradient_tail_df(const cx<float>* __restrict__ Uh,
                                                          const cx<float>* __restrict__ Ul, cx<float>* __restrict__ D,
                                                          double2* __restrict__ partial, const Geom geo, DevState* st,
                                                          int mode, double normF, double normT) {
  pdl_wait();
  if (queue_stopped(st, mode)) return;
  const int V = (int)geo.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  df fsum = {0.f, 0.f};
  float tsum = 0.f;
  if (s < V) {
    int c[4];
    site_coords_i(geo.L, s, c);
    cdf A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int st_mu = (int)geo.stride[mu];
      const int sb = c[mu] > 0 ? s - st_mu : s + (geo.L[mu] - 1) * st_mu;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const cdf own = load_cdf(Uh, Ul, (mu * 9 + q) * V + s);
        const cdf back = load_cdf(Uh, Ul, (mu * 9 + q) * V + sb);
        // sloppy double-float sums: errors ~2^-47 of the O(1) operands,
        // ~1e-14 absolute, far below what the tail resolves
        A[q].re = df_add_sloppy(A[q].re, df_add_sloppy(back.re, df_neg(own.re)));
        A[q].im = df_add_sloppy(A[q].im, df_add_sloppy(back.im, df_neg(own.im)));
        if (q == 0 || q == 4 || q == 8) fsum = df_add_sloppy(fsum, own.re);
      }
    }
    // Delta = A - A^dag - trace: off-diagonal pairs and imaginary diagonal
    const df r01 = df_add(A[1].re, df_neg(A[3].re)), i01 = df_add(A[1].im, A[3].im);
    const df r02 = df_add(A[2].re, df_neg(A[6].re)), i02 = df_add(A[2].im, A[6].im);
    const df r12 = df_add(A[5].re, df_neg(A[7].re)), i12 = df_add(A[5].im, A[7].im);
    // traceless imaginary diagonal: Im Tr A need not be small, so the
    // cancellation 2 a_k - a_l - a_m happens in double-float, before rounding
    const df a0 = A[0].im, a1 = A[4].im, a2 = A[8].im;  // times 2, below
    const df n0 = df_add(df_add({2.f * a0.h, 2.f * a0.l}, df_neg(a1)), df_neg(a2));
    const df n1 = df_add(df_add({2.f * a1.h, 2.f * a1.l}, df_neg(a0)), df_neg(a2));
    const float i0 = 2.f * (n0.h + n0.l) / 3.f, i1 = 2.f * (n1.h + n1.l) / 3.f, i2 = -(i0 + i1);
    const cx<float> d01 = mk<float>(r01.h + r01.l, i01.h + i01.l);
    const cx<float> d02 = mk<float>(r02.h + r02.l, i02.h + i02.l);
    const cx<float> d12 = mk<float>(r12.h + r12.l, i12.h + i12.l);
    D[s] = d01;
    D[V + s] = d02;
    D[2 * V + s] = d12;
    D[3 * V + s] = mk<float>(i0, i1);
    tsum = 2.f * (norm2(d01) + norm2(d02) + norm2(d12)) + i0 * i0 + i1 * i1 + i2 * i2;
  }
  // warp sums: F in double-float, theta in FP32; FP64 above the warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df other = {__shfl_down_sync(0xffffffffu, fsum.h, o), __shfl_down_sync(0xffffffffu, fsum.l, o)};
    fsum = df_add(fsum, other);
    tsum += __shfl_down_sync(0xffffffffu, tsum, o);
  }
  const double wf = fp32_to_fp64_bits(fsum.h) + fp32_to_fp64_bits(fsum.l);
  grid_reduce_warp_totals(wf, (double)tsum, partial, st, normF, normT, mode);
}

// U_mu(x) += eps(x) U + U eps(x+mu)^dag + eps(x) U eps(x+mu)^dag, the
// correction formed in FP32 from hi, added in double-float
__global__ void __launch_bounds__(256) k_tail_update_df(cx<float>* __restrict__ Uh, cx<float>* __restrict__ Ul,
                                                        const cx<float>* __restrict__ eps,
                                                        const Geom geo, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int V = (int)geo.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords_i(geo.L, s, c);
  const M3<float> ex = load_m3i<float, 9>(eps, V, s);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int st_mu = (int)geo.stride[mu];
    const int sf = c[mu] < geo.L[mu] - 1 ? s + st_mu : s - (geo.L[mu] - 1) * st_mu;
    const M3<float> ef = load_m3i<float, 9>(eps, V, sf);
    M3<float> uh;
#pragma unroll
    for (int q = 0; q < 9; ++q) uh.e[q / 3][q % 3] = Uh[(mu * 9 + q) * V + s];
    M3<float> a, d;
    mm<float, 3>(a, ex, uh);      // eps U
    mm_dag<float, 3>(d, uh, ef);  // U eps'^dag
    mm_dag_acc(d, a, ef);         // + eps U eps'^dag
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int o = (mu * 9 + q) * V + s;
      const cx<float> delta = a.e[q / 3][q % 3] + d.e[q / 3][q % 3];
      const cx<float> lo = Ul[o];
      const df re = df_add_f({uh.e[q / 3][q % 3].re, lo.re}, delta.re);
      const df im = df_add_f({uh.e[q / 3][q % 3].im, lo.im}, delta.im);
      Uh[o] = mk<float>(re.h, im.h);
      Ul[o] = mk<float>(re.l, im.l);
    }
  }
}

// double-float links -> FP64 SoA links (exact conversions, one FP64 addition)
__global__ void __launch_bounds__(256) k_df_to_fp64(const cx<float>* __restrict__ Uh, const cx<float>* __restrict__ Ul,
                                                    cx<double>* __restrict__ U, int n) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cx<float> h = ldg(Uh + i), l = ldg(Ul + i);
  U[i] = mk<double>(fp32_to_fp64_bits(h.re) + fp32_to_fp64_bits(l.re),
                    fp32_to_fp64_bits(h.im) + fp32_to_fp64_bits(l.im));
}

}  // namespace

cudaError_t launch_tail_start_df(const void* Uin64, const void* g64, void* Udf, const Geom& geo, cudaStream_t s) {
  const int64_t n = 4 * geo.V;
  auto h = static_cast<cx<float>*>(Udf);
  k_tail_start_df<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(static_cast<const cx<double>*>(Uin64),
                                                               static_cast<const cx<double>*>(g64), h, h + 36 * geo.V,
                                                               geo);
  return cudaPeekAtLastError();
}

cudaError_t launch_gradient_tail_df(const void* Udf, void* D32, double2* partial, const Geom& geo, DevState* st,
                                    int mode, cudaStream_t s) {
  auto h = static_cast<const cx<float>*>(Udf);
  const unsigned nb = (unsigned)((geo.V + 255) / 256);
  launch_pdl(k_gradient_tail_df, nb, 256, 0, s, h, h + 36 * geo.V, static_cast<cx<float>*>(D32), partial, geo, st,
             mode, 1.0 / (12.0 * (double)geo.V), 1.0 / (3.0 * (double)geo.V));
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_update_df(void* Udf, const void* eps, const Geom& geo, const DevState* st, cudaStream_t s) {
  auto h = static_cast<cx<float>*>(Udf);
  launch_pdl(k_tail_update_df, (unsigned)((geo.V + 255) / 256), 256, 0, s, h, h + 36 * geo.V,
             static_cast<const cx<float>*>(eps), geo, st);
  return cudaPeekAtLastError();
}

cudaError_t launch_df_to_fp64(const void* Udf, void* U64, int64_t V, cudaStream_t s) {
  auto h = static_cast<const cx<float>*>(Udf);
  const int64_t n = 36 * V;
  launch_pdl(k_df_to_fp64, (unsigned)((n + 255) / 256), 256, 0, s, h, h + n, static_cast<cx<double>*>(U64), (int)n);
  return cudaPeekAtLastError();
}

cudaError_t launch_gradient_tail(const void* U64, void* D32, double2* partial, const Geom& geo, DevState* st,
                                 int mode, cudaStream_t s) {
  const unsigned nb = (unsigned)((geo.V + 255) / 256);
  launch_pdl(k_gradient_tail, nb, 256, 0, s, static_cast<const cx<double>*>(U64), static_cast<cx<float>*>(D32),
             partial, geo, st, mode, 1.0 / (12.0 * (double)geo.V), 1.0 / (3.0 * (double)geo.V));
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_step(const void* D32, void* eps, int64_t V, double half_alpha, const DevState* st,
                             cudaStream_t s) {
  launch_pdl(k_tail_step, (unsigned)((V + 255) / 256), 256, 0, s, static_cast<const cx<float>*>(D32),
                                                          static_cast<cx<float>*>(eps), (int)V, (float)half_alpha,
                                                          st);
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_update(void* U64, const void* eps, const Geom& geo, const DevState* st, cudaStream_t s) {
  launch_pdl(k_tail_update, (unsigned)((geo.V + 255) / 256), 256, 0, s, static_cast<cx<double>*>(U64),
                                                                  static_cast<const cx<float>*>(eps), geo, st);
  return cudaPeekAtLastError();
}

}  // namespace lgf
