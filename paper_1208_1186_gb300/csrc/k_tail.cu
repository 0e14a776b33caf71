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
// Gram-Schmidt) to ~0.3k (sums), which is what the FP64 pipe of this GPU
// (1/62 of FP32) can afford.
#include "lgf_kernels.cuh"
#include "lgf_reduce.cuh"

namespace lgf {

namespace {

__global__ void __launch_bounds__(256) k_gradient_tail(const cx<double>* __restrict__ U, cx<float>* __restrict__ D,
                                                       double2* __restrict__ partial, const Geom geo, DevState* st,
                                                       int mode, double normF, double normT) {
  pdl_wait();
  if (mode == 1 && st->done) return;
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

}  // namespace

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
