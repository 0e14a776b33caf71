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
// That is tail mode 2.  FP64 work per site drops from ~2.5k operations (FP64
// products, FFT, Gram-Schmidt) to ~0.3k (sums), yet even those sums bound the
// kernels on this GPU, whose FP64 pipe runs at 1/62 of FP32.  The default tail
// (mode 0) does every operation on the FP32 pipe instead, in double-float form
// where the precision is needed: two FP32 numbers per real, value = hi + lo
// with |lo| <= ulp(hi)/2 (48 significant bits), handled by error-free
// transformations (Knuth's two-sum, Dekker's fast-two-sum, the FMA
// two-product; lgf_df.cuh).  It also runs in gauge representation: the links
// of the tail start stay fixed and the tail accumulates its own gauge
// transformation 1 + eta(x), close to the identity:
//
//   k_promote_df        the FP32 gauge G reunitarised in double-float
//                       (Gram-Schmidt), stored as hi and lo planes;
//   k_tail_start_df     U = g U_loaded g(x+mu)^dag from the FP64 input (split
//                       exactly into hi + lo by bit manipulation) and that
//                       g, products in double-float;
//   k_tail_base         Delta(U) and each site's F term, once (Delta is linear
//                       in the link sums, so the tail's gradient is this
//                       fixed part plus that of the corrections);
//   k_gradient_tail_eta Delta of the current links (1 + eta) U (1 + eta')^dag:
//                       the fixed part plus the FP32 corrections, F summed
//                       in double-float per warp, D stored as FP32;
//   k_tail_eta_step     eps from the accelerated gradient, 1 + eta <-
//                       (1 + eps)(1 + eta) at each site in double-float, X
//                       added exactly (no link is rewritten);
//   k_tail_apply_eta,   the links as FP64 planes, for the calls that need
//   k_df_to_fp64        them; otherwise the host store forms them in FP64
//                       directly (k_store_aos_df).
//
// The corrections' FP32 rounding (2^-24 |eta| < 1e-12) perturbs only the
// gradient that the tail drives to zero; the links and 1 + eta are formed
// to ~2^-47.
#include "lgf_df.cuh"
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

// eps = X + X^2 / 2, X = h Delta~ (traceless anti-Hermitian), from the
// packed accelerated gradient c0..c3 (Delta~_01, Delta~_02, Delta~_12,
// Im Delta~_00 + i Im Delta~_11)
__device__ __forceinline__ M3<float> tail_eps(cx<float> c0, cx<float> c1, cx<float> c2, cx<float> c3, float h) {
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
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) X.e[i][j] = X.e[i][j] + scale(X2.e[i][j], 0.5f);
  return X;
}

// eps as 9 FP32 planes (the FP64-link tail)
__global__ void __launch_bounds__(256) k_tail_step(const cx<float>* __restrict__ D, cx<float>* __restrict__ eps,
                                                   int V, float h, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const M3<float> e = tail_eps(ldg(D + s), ldg(D + V + s), ldg(D + 2 * V + s), ldg(D + 3 * V + s), h);
#pragma unroll
  for (int q = 0; q < 9; ++q) eps[q * V + s] = e.e[q / 3][q % 3];
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

// G reunitarised in double-float: Gram-Schmidt on its first two rows (the
// projection the iteration uses, Sec. 2.1), row 3 the conjugated cross
// product, so that Gh + Gl is special unitary to ~2^-47.  The FP32 G is
// within ~1e-6 of unitary, so the row norms are 1 + O(1e-6) and the
// reciprocal square root is the first-order-corrected rsqrtf of df_rsqrt.
// Input: rows 0 and 1 of G (the first 6 planes of either storage form).
// Output: Gh and Gl, each 9 complex FP32 planes.
__global__ void __launch_bounds__(256) k_promote_df(const cx<float>* __restrict__ G, cx<float>* __restrict__ gh,
                                                    cx<float>* __restrict__ gl, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  cx<float> r0[3], r1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r0[j] = ldg(G + j * V + s);
    r1[j] = ldg(G + (3 + j) * V + s);
  }
  // row 0 / |row 0|
  dacc n = dacc_zero();
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dacc_prod(n, r0[j].re, r0[j].re);
    dacc_prod(n, r0[j].im, r0[j].im);
  }
  const df inv0 = df_rsqrt(dacc_result(n));
  cdf u[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) u[j] = {df_mul_f(inv0, r0[j].re), df_mul_f(inv0, r0[j].im)};
  // <u, row 1> = sum conj(u_j) r1_j
  dacc pr = dacc_zero(), pi = dacc_zero();
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dacc_prod_df(pr, u[j].re, r1[j].re);
    dacc_prod_df(pr, u[j].im, r1[j].im);
    dacc_prod_df(pi, u[j].re, r1[j].im);
    dacc_prod_df(pi, df_neg(u[j].im), r1[j].re);
  }
  const df ipr = dacc_result(pr), ipi = dacc_result(pi);
  // w = row 1 - <u, row 1> u, then w / |w|
  cdf w[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dacc a = {r1[j].re, 0.f}, b = {r1[j].im, 0.f};
    dacc_prod_dd(a, df_neg(ipr), u[j].re);
    dacc_prod_dd(a, ipi, u[j].im);
    dacc_prod_dd(b, df_neg(ipr), u[j].im);
    dacc_prod_dd(b, df_neg(ipi), u[j].re);
    w[j] = {dacc_result(a), dacc_result(b)};
  }
  n = dacc_zero();
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dacc_prod_dd(n, w[j].re, w[j].re);
    dacc_prod_dd(n, w[j].im, w[j].im);
  }
  const df inv1 = df_rsqrt(dacc_result(n));
#pragma unroll
  for (int j = 0; j < 3; ++j) w[j] = {df_mul(w[j].re, inv1), df_mul(w[j].im, inv1)};
  // row 2 = conj(u x w): v_j = conj(u_k w_l - u_l w_k), (j, k, l) cyclic
  cdf v[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3, l = (j + 2) % 3;
    dacc a = dacc_zero(), b = dacc_zero();
    dacc_prod_dd(a, u[k].re, w[l].re);
    dacc_prod_dd(a, df_neg(u[k].im), w[l].im);
    dacc_prod_dd(a, df_neg(u[l].re), w[k].re);
    dacc_prod_dd(a, u[l].im, w[k].im);
    // -Im(u_k w_l - u_l w_k)
    dacc_prod_dd(b, df_neg(u[k].re), w[l].im);
    dacc_prod_dd(b, df_neg(u[k].im), w[l].re);
    dacc_prod_dd(b, u[l].re, w[k].im);
    dacc_prod_dd(b, u[l].im, w[k].re);
    v[j] = {dacc_result(a), dacc_result(b)};
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    gh[j * V + s] = mk<float>(u[j].re.h, u[j].im.h);
    gl[j * V + s] = mk<float>(u[j].re.l, u[j].im.l);
    gh[(3 + j) * V + s] = mk<float>(w[j].re.h, w[j].im.h);
    gl[(3 + j) * V + s] = mk<float>(w[j].re.l, w[j].im.l);
    gh[(6 + j) * V + s] = mk<float>(v[j].re.h, v[j].im.h);
    gl[(6 + j) * V + s] = mk<float>(v[j].re.l, v[j].im.l);
  }
}

// The gauge transformation that a double-float tail has applied to the
// loaded links, (1 + eta)(Gh + Gl), as FP64 [s][3][3] complex: both factors
// formed exactly in FP64 from their FP32 parts, the product in FP64.
__global__ void __launch_bounds__(256) k_store_gauge_df(const cx<float>* __restrict__ gh,
                                                        const cx<float>* __restrict__ gl,
                                                        const cx<float>* __restrict__ eh,
                                                        const cx<float>* __restrict__ el, double* __restrict__ out,
                                                        int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  M3<double> E, Gd, R;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const cx<float> a = ldg(gh + q * V + s), b = ldg(gl + q * V + s);
    const cx<float> c = ldg(eh + q * V + s), d = ldg(el + q * V + s);
    Gd.e[q / 3][q % 3] = mk<double>((double)a.re + (double)b.re, (double)a.im + (double)b.im);
    E.e[q / 3][q % 3] = mk<double>((q % 4 == 0 ? 1.0 : 0.0) + ((double)c.re + (double)d.re), (double)c.im + (double)d.im);
  }
  mm<double, 3>(R, E, Gd);
  double2* o = reinterpret_cast<double2*>(out + (size_t)s * 18);
#pragma unroll
  for (int q = 0; q < 9; ++q) o[q] = make_double2(R.e[q / 3][q % 3].re, R.e[q / 3][q % 3].im);
}

// U_mu(x) = g(x) U_loaded,mu(x) g(x+mu)^dag, one thread per (site, mu), with
// g = Gh + Gl from k_promote_df and U = Uh + Ul the exact split of the FP64
// input.  Row a of W = g U: Gh Uh by compensated dot products of exact FP32
// products, the first-order terms Gl Uh + Gh Ul (~2^-24 of the result) added
// to the low parts.  Then row a of W g'^dag the same way: W Fh'^dag with W in
// double-float, plus Wh Fl'^dag in the low parts.  The dropped second-order
// terms are ~2^-48.  Rows are processed one at a time (no unrolling) so that
// a thread holds U and one row of g and W, not all three.
__global__ void __launch_bounds__(128, 4) k_tail_start_df(const cx<double>* __restrict__ Uin,
                                                          const cx<float>* __restrict__ gh,
                                                          const cx<float>* __restrict__ gl, cx<float>* __restrict__ Uh,
                                                          cx<float>* __restrict__ Ul, const Geom geo) {
  const int V = (int)geo.V;
  // a block is 32 consecutive sites x the 4 directions, one warp per
  // direction: the warps share g(x) through L1
  const int mu = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + (threadIdx.x & 31);
  if (s >= V) return;
  int c[4];
  site_coords_i(geo.L, s, c);
  // selects, not a runtime index: keeps c and the geometry in registers
  const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
  const int Lm = mu == 0 ? geo.L[0] : mu == 1 ? geo.L[1] : mu == 2 ? geo.L[2] : geo.L[3];
  const int st_mu = mu == 0 ? 1 : mu == 1 ? geo.L[0] : mu == 2 ? geo.L[0] * geo.L[1] : geo.L[0] * geo.L[1] * geo.L[2];
  const int sf = cm < Lm - 1 ? s + st_mu : s - (Lm - 1) * st_mu;
  cx<float> UH[9], UL[9];
  split_matrix(Uin + mu * 9 * V, V, s, UH, UL);
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    cx<float> xh[3], xl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      xh[k] = ldg(gh + (a * 3 + k) * V + s);
      xl[k] = ldg(gl + (a * 3 + k) * V + s);
    }
    cdf W[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dacc re = dacc_zero(), im = dacc_zero();
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cx<float> x = xh[k], y = UH[k * 3 + b], xe = xl[k], ye = UL[k * 3 + b];
        dacc_prod(re, x.re, y.re);
        dacc_prod(re, -x.im, y.im);
        dacc_prod(im, x.re, y.im);
        dacc_prod(im, x.im, y.re);
        dacc_lo(re, xe.re, y.re);
        dacc_lo(re, -xe.im, y.im);
        dacc_lo(re, x.re, ye.re);
        dacc_lo(re, -x.im, ye.im);
        dacc_lo(im, xe.re, y.im);
        dacc_lo(im, xe.im, y.re);
        dacc_lo(im, x.re, ye.im);
        dacc_lo(im, x.im, ye.re);
      }
      W[b] = {dacc_result(re), dacc_result(im)};
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dacc re = dacc_zero(), im = dacc_zero();
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // W conj(F): re += W.re F.re + W.im F.im, im += W.im F.re - W.re F.im
        const cx<float> f = ldg(gh + (b * 3 + k) * V + sf), fe = ldg(gl + (b * 3 + k) * V + sf);
        const cdf w = W[k];
        dacc_prod_df(re, w.re, f.re);
        dacc_prod_df(re, w.im, f.im);
        dacc_prod_df(im, w.im, f.re);
        dacc_prod_df(im, df_neg(w.re), f.im);
        dacc_lo(re, w.re.h, fe.re);
        dacc_lo(re, w.im.h, fe.im);
        dacc_lo(im, w.im.h, fe.re);
        dacc_lo(im, -w.re.h, fe.im);
      }
      const df r = dacc_result(re), m = dacc_result(im);
      const int o = (mu * 9 + a * 3 + b) * V + s;
      Uh[o] = mk<float>(r.h, m.h);
      Ul[o] = mk<float>(r.l, m.l);
    }
  }
}

// a += v (double-float) by one exact two-sum; v's low part and the sum
// error go to the low part (the Dot2 accumulation of lgf_df.cuh for sums)
__device__ __forceinline__ void dacc_add(dacc& a, float vh, float vl) {
  const df t = two_sum(a.h, vh);
  a.h = t.h;
  a.l = __fadd_rn(a.l, __fadd_rn(vl, t.l));
}

// ---------------------------------------------------------------------------
// The tail in gauge representation.  The double-float links U of the tail
// start stay fixed; the tail accumulates a gauge transformation 1 + eta(x)
// close to the identity (eta FP32, |eta| ~ 1e-5), so that its current links
// are
//   U'_mu(x) = (1 + eta(x)) U_mu(x) (1 + eta(x+mu))^dag
//            = U + eta U + U eta'^dag + eta U eta'^dag,
// the correction (all terms) formed in FP32 from hi and added in double-float.
// The update of the method, U' <- g U' g(x+mu)^dag with g = 1 + eps, becomes
// 1 + eta <- (1 + eps)(1 + eta) at each site alone; no link is written.
// The FP32 rounding of each correction (|eps| 2^-24 per step) is that of
// the link-update form of the defect correction.
// ---------------------------------------------------------------------------

// a += v for an FP32 v, exactly (one two-sum)
__device__ __forceinline__ void dacc_add_f(dacc& a, float v) { dacc_add(a, v, 0.f); }

// The fixed part of the tail's gradient.  Delta is linear in A = sum_mu
// U'_mu(x-mu) - U'_mu(x), and U' = U + (small corrections), so Delta(U') =
// Delta(U) + Delta(corrections) with Delta(U) fixed for the whole tail.
// This kernel forms Delta(U) (~1e-6 after the FP32 phase) by double-float
// sums and stores it packed in FP32 (error ~2^-24 1e-6, below the FP32
// rounding of the corrections), and each site's F term sum_mu Re tr U_mu(x)
// in double-float.  Once per tail start.
__global__ void __launch_bounds__(256, 2) k_tail_base(const cx<float>* __restrict__ Uh, const cx<float>* __restrict__ Ul,
                                                      cx<float>* __restrict__ D0, float2* __restrict__ F0,
                                                      const Geom geo) {
  pdl_wait();
  const int V = (int)geo.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords_i(geo.L, s, c);
  dacc Ar[9], Ai[9], fs = dacc_zero();
#pragma unroll
  for (int q = 0; q < 9; ++q) Ar[q] = Ai[q] = dacc_zero();
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int st_mu = (int)geo.stride[mu];
    const int sb = c[mu] > 0 ? s - st_mu : s + (geo.L[mu] - 1) * st_mu;
    cx<float> oh[9], ol[9], bh[9], bl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int o = (mu * 9 + q) * V;
      oh[q] = ldg(Uh + o + s);
      ol[q] = ldg(Ul + o + s);
      bh[q] = ldg(Uh + o + sb);
      bl[q] = ldg(Ul + o + sb);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      dacc_add(Ar[q], bh[q].re, bl[q].re);
      dacc_add(Ar[q], -oh[q].re, -ol[q].re);
      dacc_add(Ai[q], bh[q].im, bl[q].im);
      dacc_add(Ai[q], -oh[q].im, -ol[q].im);
      if (q == 0 || q == 4 || q == 8) dacc_add(fs, oh[q].re, ol[q].re);
    }
  }
  df A_re[9], A_im[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    A_re[q] = dacc_result(Ar[q]);
    A_im[q] = dacc_result(Ai[q]);
  }
  // Delta = A - A^dag - trace: off-diagonal pairs and imaginary diagonal
  const df r01 = df_add(A_re[1], df_neg(A_re[3])), i01 = df_add(A_im[1], A_im[3]);
  const df r02 = df_add(A_re[2], df_neg(A_re[6])), i02 = df_add(A_im[2], A_im[6]);
  const df r12 = df_add(A_re[5], df_neg(A_re[7])), i12 = df_add(A_im[5], A_im[7]);
  // traceless imaginary diagonal: Im Tr A need not be small, so the
  // cancellation 2 a_k - a_l - a_m happens in double-float, before rounding
  const df a0 = A_im[0], a1 = A_im[4], a2 = A_im[8];
  const df n0 = df_add(df_add({2.f * a0.h, 2.f * a0.l}, df_neg(a1)), df_neg(a2));
  const df n1 = df_add(df_add({2.f * a1.h, 2.f * a1.l}, df_neg(a0)), df_neg(a2));
  D0[s] = mk<float>(r01.h + r01.l, i01.h + i01.l);
  D0[V + s] = mk<float>(r02.h + r02.l, i02.h + i02.l);
  D0[2 * V + s] = mk<float>(r12.h + r12.l, i12.h + i12.l);
  D0[3 * V + s] = mk<float>(2.f * (n0.h + n0.l) / 3.f, 2.f * (n1.h + n1.l) / 3.f);
  const df f = dacc_result(fs);
  F0[s] = make_float2(f.h, f.l);
}

// Delta and F/theta of U' = U + corrections: the fixed part from k_tail_base,
// the corrections from the FP32 hi links and eta (hi).  Backward links
// first: P = sum eta(x-mu) U_mu(x-mu) and T = sum (U + P terms), closed by
// one product T eta(x)^dag; then the forward links: W = sum U eta'^dag and
// T = sum (U + W terms), closed by eta(x) T.  Ten FP32 products per site.
__global__ void __launch_bounds__(256, 2) k_gradient_tail_eta(const cx<float>* __restrict__ Uh,
                                                              const cx<float>* __restrict__ eta,
                                                              const cx<float>* __restrict__ D0,
                                                              const float2* __restrict__ F0,
                                                              cx<float>* __restrict__ D, double2* __restrict__ partial,
                                                              const Geom geo, DevState* st, int mode, double normF,
                                                              double normT) {
  pdl_wait();
  if (queue_stopped(st, mode)) return;
  const int V = (int)geo.V;
  // a grid-stride loop over sites (2 CTAs per SM): each thread adds its
  // sites' F terms in double-float and their theta terms in compensated
  // FP32; the block and grid sums run once per CTA
  df fsum = {0.f, 0.f};
  float tsum = 0.f, tcomp = 0.f;
  const int stride = gridDim.x * blockDim.x;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += stride) {
    int c[4];
    site_coords_i(geo.L, s, c);
    M3<float> Cc, T;  // the links' corrections; the pending factor of one product
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Cc.e[i][j] = T.e[i][j] = mk<float>(0.f, 0.f);
    // backward links (1 + eta(x-mu)) U (1 + eta(x))^dag
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int st_mu = (int)geo.stride[mu];
      const int sb = c[mu] > 0 ? s - st_mu : s + (geo.L[mu] - 1) * st_mu;
      M3<float> ub, eb;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        ub.e[q / 3][q % 3] = ldg(Uh + (mu * 9 + q) * V + sb);
        eb.e[q / 3][q % 3] = ldg(eta + q * V + sb);
      }
      M3<float> y;
      mm<float, 3>(y, eb, ub);  // eta(x-mu) U
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          Cc.e[i][j] = Cc.e[i][j] + y.e[i][j];
          T.e[i][j] = T.e[i][j] + (ub.e[i][j] + y.e[i][j]);
        }
    }
    {
      const M3<float> ex = load_m3i<float, 9>(eta, V, s);
      mm_dag_acc(Cc, T, ex);  // + sum (1 + eta(x-mu)) U eta(x)^dag
    }
    // forward links (1 + eta(x)) U (1 + eta(x+mu))^dag
    float fc = 0.f;  // Re tr of their corrections
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) T.e[i][j] = mk<float>(0.f, 0.f);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int st_mu = (int)geo.stride[mu];
      const int sf = c[mu] < geo.L[mu] - 1 ? s + st_mu : s - (geo.L[mu] - 1) * st_mu;
      M3<float> uf, ef;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        uf.e[q / 3][q % 3] = ldg(Uh + (mu * 9 + q) * V + s);
        ef.e[q / 3][q % 3] = ldg(eta + q * V + sf);
      }
      M3<float> w;
      mm_dag<float, 3>(w, uf, ef);  // U eta(x+mu)^dag
      fc += w.e[0][0].re + w.e[1][1].re + w.e[2][2].re;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          Cc.e[i][j] = Cc.e[i][j] - w.e[i][j];
          T.e[i][j] = T.e[i][j] + (uf.e[i][j] + w.e[i][j]);
        }
    }
    {
      const M3<float> ex = load_m3i<float, 9>(eta, V, s);
      M3<float> m;
      mm<float, 3>(m, ex, T);  // eta(x) sum U (1 + eta(x+mu))^dag
      fc += m.e[0][0].re + m.e[1][1].re + m.e[2][2].re;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Cc.e[i][j] = Cc.e[i][j] - m.e[i][j];
    }
    // Delta = Delta(U) + Delta(corrections)
    const cx<float> b01 = ldg(D0 + s), b02 = ldg(D0 + V + s), b12 = ldg(D0 + 2 * V + s), bd = ldg(D0 + 3 * V + s);
    const cx<float> d01 = b01 + (Cc.e[0][1] - conj(Cc.e[1][0]));
    const cx<float> d02 = b02 + (Cc.e[0][2] - conj(Cc.e[2][0]));
    const cx<float> d12 = b12 + (Cc.e[1][2] - conj(Cc.e[2][1]));
    const float c0 = 2.f * Cc.e[0][0].im, c1 = 2.f * Cc.e[1][1].im, c2 = 2.f * Cc.e[2][2].im;
    const float ctr = (c0 + c1 + c2) / 3.f;
    const float i0 = bd.re + (c0 - ctr), i1 = bd.im + (c1 - ctr), i2 = -(i0 + i1);
    D[s] = d01;
    D[V + s] = d02;
    D[2 * V + s] = d12;
    D[3 * V + s] = mk<float>(i0, i1);
    const float ts = 2.f * (norm2(d01) + norm2(d02) + norm2(d12)) + i0 * i0 + i1 * i1 + i2 * i2;
    {  // Kahan-compensated theta terms
      const float y = ts - tcomp;
      const float t = tsum + y;
      tcomp = (t - tsum) - y;
      tsum = t;
    }
    const float2 f0 = __ldg(F0 + s);
    dacc fs = {f0.x, f0.y};
    dacc_add_f(fs, fc);
    fsum = df_add(fsum, dacc_result(fs));
  }
  tsum -= tcomp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df other = {__shfl_down_sync(0xffffffffu, fsum.h, o), __shfl_down_sync(0xffffffffu, fsum.l, o)};
    fsum = df_add(fsum, other);
    tsum += __shfl_down_sync(0xffffffffu, tsum, o);
  }
  const double wf = fp32_to_fp64_bits(fsum.h) + fp32_to_fp64_bits(fsum.l);
  grid_reduce_warp_totals(wf, (double)tsum, partial, st, normF, normT, mode);
}

// 1 + eta <- (1 + eps)(1 + eta) at every site (tail_eta_site, lgf_df.cuh),
// from the accelerated gradient in global memory; where the plane pipeline
// applies, the same step is fused with the inverse x-y transform instead
// (k_plane_xyinv_eta).
__global__ void __launch_bounds__(128, 5) k_tail_eta_step(const cx<float>* __restrict__ D, cx<float>* __restrict__ eh,
                                                       cx<float>* __restrict__ el, int V, float h,
                                                       const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  tail_eta_site(ldg(D + s), ldg(D + V + s), ldg(D + 2 * V + s), ldg(D + 3 * V + s), h, eh, el, V, s);
}

// U <- U' (the caller then clears eta): one thread per (site, direction), a
// block 32 sites x 4 directions
__global__ void __launch_bounds__(128) k_tail_apply_eta(cx<float>* __restrict__ Uh, cx<float>* __restrict__ Ul,
                                                        const cx<float>* __restrict__ eh,
                                                        const cx<float>* __restrict__ el, const Geom geo) {
  pdl_wait();
  const int V = (int)geo.V;
  const int mu = threadIdx.x >> 5;
  const int s = blockIdx.x * 32 + (threadIdx.x & 31);
  if (s >= V) return;
  int c[4];
  site_coords_i(geo.L, s, c);
  const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
  const int Lm = mu == 0 ? geo.L[0] : mu == 1 ? geo.L[1] : mu == 2 ? geo.L[2] : geo.L[3];
  const int st_mu = mu == 0 ? 1 : mu == 1 ? geo.L[0] : mu == 2 ? geo.L[0] * geo.L[1] : geo.L[0] * geo.L[1] * geo.L[2];
  const int sf = cm < Lm - 1 ? s + st_mu : s - (Lm - 1) * st_mu;
  const M3<float> xh = load_m3i<float, 9>(eh, V, s), xl = load_m3i<float, 9>(el, V, s);
  const M3<float> fh = load_m3i<float, 9>(eh, V, sf), fl = load_m3i<float, 9>(el, V, sf);
  M3<float> uh;
  cx<float> ul[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int o = (mu * 9 + q) * V + s;
    uh.e[q / 3][q % 3] = Uh[o];
    ul[q] = Ul[o];
  }
  df re[9], im[9];
  tail_link_exact(uh, ul, xh, xl, fh, fl, re, im);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int o = (mu * 9 + q) * V + s;
    Uh[o] = mk<float>(re[q].h, im[q].h);
    Ul[o] = mk<float>(re[q].l, im[q].l);
  }
}

// double-float links -> FP64 SoA links (exact conversions, one FP64 addition)
__global__ void __launch_bounds__(256) k_df_to_fp64(const cx<float>* __restrict__ Uh, const cx<float>* __restrict__ Ul,
                                                    cx<double>* __restrict__ U, int n) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cx<float> h = ldg(Uh + i), l = ldg(Ul + i);
  U[i] = mk<double>(df_to_double(h.re, l.re), df_to_double(h.im, l.im));
}

}  // namespace

cudaError_t launch_store_gauge_df(const void* g_df, const void* eta, int64_t V, double* out, cudaStream_t s) {
  auto g = static_cast<const cx<float>*>(g_df);
  auto e = static_cast<const cx<float>*>(eta);
  k_store_gauge_df<<<(unsigned)((V + 255) / 256), 256, 0, s>>>(g, g + 9 * V, e, e + 9 * V, out, (int)V);
  return cudaPeekAtLastError();
}

cudaError_t launch_promote_df(const void* G32, void* g_df, int64_t V, cudaStream_t s) {
  auto h = static_cast<cx<float>*>(g_df);
  k_promote_df<<<(unsigned)((V + 255) / 256), 256, 0, s>>>(static_cast<const cx<float>*>(G32), h, h + 9 * V, (int)V);
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_start_df(const void* Uin64, const void* g_df, void* Udf, const Geom& geo, cudaStream_t s) {
  auto h = static_cast<cx<float>*>(Udf);
  auto g = static_cast<const cx<float>*>(g_df);
  k_tail_start_df<<<(unsigned)((geo.V + 31) / 32), 128, 0, s>>>(static_cast<const cx<double>*>(Uin64), g,
                                                               g + 9 * geo.V, h, h + 36 * geo.V, geo);
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_base(const void* Udf, void* base, const Geom& geo, cudaStream_t s) {
  auto h = static_cast<const cx<float>*>(Udf);
  auto D0 = static_cast<cx<float>*>(base);
  launch_pdl(k_tail_base, (unsigned)((geo.V + 255) / 256), 256, 0, s, h, h + 36 * geo.V, D0,
             reinterpret_cast<float2*>(D0 + 4 * geo.V), geo);
  return cudaPeekAtLastError();
}

// the tail gradient's grid: 2 CTAs per SM (grid-stride), or one site per thread
constexpr bool kTailGridStride = true;

static int tail_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, m = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || m <= 0)
      return 1;
    n = m;
  }
  return n;
}

cudaError_t launch_gradient_tail_eta(const void* Udf, const void* eta, const void* base, void* D32,
                                     double2* partial, const Geom& geo, DevState* st, int mode, cudaStream_t s) {
  auto D0 = static_cast<const cx<float>*>(base);
  const int64_t full = (geo.V + 255) / 256;
  const int64_t cap = 2 * (int64_t)tail_sm_count();
  const unsigned nb = (unsigned)(kTailGridStride && full > cap ? cap : full);
  launch_pdl(k_gradient_tail_eta, nb, 256, 0, s, static_cast<const cx<float>*>(Udf),
             static_cast<const cx<float>*>(eta), D0, reinterpret_cast<const float2*>(D0 + 4 * geo.V),
             static_cast<cx<float>*>(D32), partial, geo, st, mode, 1.0 / (12.0 * (double)geo.V),
             1.0 / (3.0 * (double)geo.V));
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_eta_step(const void* D32, void* eta, int64_t V, double half_alpha, const DevState* st,
                                 cudaStream_t s) {
  auto e = static_cast<cx<float>*>(eta);
  launch_pdl(k_tail_eta_step, (unsigned)((V + 127) / 128), 128, 0, s, static_cast<const cx<float>*>(D32), e,
             e + 9 * V, (int)V, (float)half_alpha, st);
  return cudaPeekAtLastError();
}

cudaError_t launch_tail_apply_eta(void* Udf, void* eta, const Geom& geo, cudaStream_t s) {
  auto h = static_cast<cx<float>*>(Udf);
  auto e = static_cast<const cx<float>*>(eta);
  launch_pdl(k_tail_apply_eta, (unsigned)((geo.V + 31) / 32), 128, 0, s, h, h + 36 * geo.V, e, e + 9 * geo.V, geo);
  cudaError_t err = cudaPeekAtLastError();
  if (err != cudaSuccess) return err;
  return cudaMemsetAsync(eta, 0, (size_t)18 * geo.V * sizeof(cx<float>), s);
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
