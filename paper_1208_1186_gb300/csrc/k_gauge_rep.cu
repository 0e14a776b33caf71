// FP32 engine in gauge representation.
//
// Steepest descent only ever moves the links along their gauge orbit: after n
// iterations U_mu(x) = G(x) U0_mu(x) G(x+mu)^dagger, with U0 the loaded links
// and G = g_n ... g_1 the accumulated gauge transformation.  This engine
// keeps U0 fixed and updates G instead of the links: the update of the method,
// U_mu(x) <- g(x) U_mu(x) g(x+mu)^dagger, becomes G(x) <- g(x) G(x), and the
// gradient kernel forms the current links on the fly.  Per iteration the link
// array is read once and never written, which removes the link write-back
// and the separate update sweep (about 570 instead of 1420 algorithmic bytes
// per site for 18-real FP32 storage), and the links can never drift off the
// orbit of the loaded configuration.  The FP64 tail starts from
// G U0 G^dagger formed in FP64 from the FP64 input.
//
//   k_gradient_grep  B = sum_mu G(x-mu) U0_mu(x-mu),  C = sum_mu U0_mu(x) G(x+mu)^dag,
//                    sum_mu U_mu(x) = G(x) C,  sum_mu U_mu(x-mu) = B G(x)^dag,
//                    A = B G^dag - G C, then Delta, F, theta as in k_gradient
//                    (10 SU(3) products per site instead of 16).
//   k_gstep          g = reunitarised (1 + alpha/2 Delta~) (or the reunitarised exact
//                    exponential), G <- reunitarised g G.
//   k_materialize    G(x) U0_mu(x) G(x+mu)^dag as host-layout FP64 links.
#include "lgf_gstep.cuh"
#include "lgf_kernels.cuh"
#include "lgf_reduce.cuh"

namespace lgf {

namespace {

template <class T>
__device__ __forceinline__ void add_to(M3<T>& acc, const M3<T>& t) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc.e[i][j] = acc.e[i][j] + t.e[i][j];
}

template <class T, int NC>
__device__ __forceinline__ M3<T> load_rw(const cx<T>* base, int64_t V, int64_t s) {
  M3<T> m;
#pragma unroll
  for (int c = 0; c < NC; ++c) m.e[c / 3][c % 3] = base[c * V + s];
  if (NC == 6) complete_row3(m);
  return m;
}

// Grid-stride loop over sites with two CTAs per SM: each thread sums its
// sites' F and theta terms in FP32 with Kahan compensation (relative error
// ~1e-7 of the thread's sum however many sites it takes; FP64 conversions
// and additions per site cost 6% of this kernel on GB300), warps and above
// in FP64, and the block reduction (two barriers) runs once per CTA instead
// of once per 256 sites.  The site-to-thread map and the summation order are
// fixed by the grid, so results are reproducible.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// The per-site work of k_gradient_grep: Delta(x) stored packed, the F and
// theta terms added to the thread's compensated sums.
template <class T, int NC>
__device__ __forceinline__ void grep_site(const cx<T>* __restrict__ U0, const cx<T>* __restrict__ G,
                                          cx<T>* __restrict__ D, const Geom& geo, int V, int s, const int c[4],
                                          T& fs, T& fc, T& ts, T& tc) {
  M3<T> B, C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) B.e[i][j] = C.e[i][j] = mk<T>(0, 0);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const cx<T>* base = U0 + mu * NC * V;
    const int st_mu = (int)geo.stride[mu];
    const int span = (geo.L[mu] - 1) * st_mu;
    {
      const int sf = c[mu] < geo.L[mu] - 1 ? s + st_mu : s - span;
      const M3<T> u = load_m3i<T, NC>(base, V, s);
      const M3<T> gf = load_m3i<T, NC>(G, V, sf);
      mm_dag_acc(C, u, gf);
    }
    {
      const int sb = c[mu] > 0 ? s - st_mu : s + span;
      const M3<T> gb = load_m3i<T, NC>(G, V, sb);
      const M3<T> ub = load_m3i<T, NC>(base, V, sb);
      mm_acc(B, gb, ub);
    }
  }
  const M3<T> gx = load_m3i<T, NC>(G, V, s);
  M3<T> Uf, Ub;
  mm<T, 3>(Uf, gx, C);      // sum of the links leaving x
  mm_dag<T, 3>(Ub, B, gx);  // sum of the links arriving at x
  const T fsum = Uf.e[0][0].re + Uf.e[1][1].re + Uf.e[2][2].re;
  M3<T> A;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A.e[i][j] = Ub.e[i][j] - Uf.e[i][j];
  const cx<T> d01 = A.e[0][1] - conj(A.e[1][0]);
  const cx<T> d02 = A.e[0][2] - conj(A.e[2][0]);
  const cx<T> d12 = A.e[1][2] - conj(A.e[2][1]);
  const T a0 = 2 * A.e[0][0].im, a1 = 2 * A.e[1][1].im, a2 = 2 * A.e[2][2].im;
  const T tr = (a0 + a1 + a2) / (T)3;
  const T i0 = a0 - tr, i1 = a1 - tr, i2 = -(i0 + i1);
  D[s] = d01;
  D[V + s] = d02;
  D[2 * V + s] = d12;
  D[3 * V + s] = mk<T>(i0, i1);
  const T tsum = 2 * (norm2(d01) + norm2(d02) + norm2(d12)) + i0 * i0 + i1 * i1 + i2 * i2;
  kahan_add(fs, fc, fsum);
  kahan_add(ts, tc, tsum);
}

template <class T, int NC>
__global__ void __launch_bounds__(kGrepThreads, 2) k_gradient_grep(const cx<T>* __restrict__ U0,
                                                                const cx<T>* __restrict__ G, cx<T>* __restrict__ D,
                                                                double2* __restrict__ partial, const Geom geo,
                                                                DevState* st, int mode, double normF, double normT) {
  pdl_wait();
  if (queue_stopped(st, mode)) return;
  const int V = (int)geo.V;  // 36 V < 2^31 for extents <= 64
  T fs = 0, fc = 0, ts = 0, tc = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += stride) {
    int c[4];
    site_coords_r(geo, s, c);
    grep_site<T, NC>(U0, G, D, geo, V, s, c, fs, fc, ts, tc);
  }
  grid_reduce<T>(fs - fc, ts - tc, partial, st, normF, normT, mode);
}

// g from the accelerated gradient; G <- g G unless G is null; g stored if
// g_out is not null.  RT: arithmetic of g, the product and both projections.
template <class T, int NC, class RT, bool EXACT>
__global__ void __launch_bounds__(256) k_gstep(const cx<T>* __restrict__ D, cx<T>* G, cx<T>* __restrict__ g_out,
                                               int64_t V, double hd, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  gstep_site<T, NC, RT>(ldg(D + s), ldg(D + V + s), ldg(D + 2 * V + s), ldg(D + 3 * V + s), (RT)hd, G, g_out, V, s,
                        EXACT);
}

// one thread per (site, mu): the current link G(x) U0 G(x+mu)^dag in the host
// layout, staged through shared memory like k_store_aos (the AoS side may be
// host memory the device writes directly)
template <class T, int NC>
__global__ void __launch_bounds__(kStageMats) k_materialize(const cx<T>* __restrict__ U0, const cx<T>* __restrict__ G,
                                                            double* __restrict__ aos, const Geom geo) {
  __shared__ double sm[kStageMats * kStagePitch];
  const int64_t V = geo.V;
  const int64_t first = (int64_t)blockIdx.x * kStageMats;
  const int n = (int)(4 * V - first < kStageMats ? 4 * V - first : kStageMats);
  if ((int)threadIdx.x < n) {
    const int64_t i = first + threadIdx.x;
    const int64_t s = i >> 2;
    const int mu = (int)(i & 3);
    int c[4];
    site_coords(geo, s, c);
    const M3<T> u = load_m3<T, NC>(U0 + (int64_t)mu * NC * V, V, s);
    const M3<T> gx = load_m3<T, NC>(G, V, s);
    const M3<T> gf = load_m3<T, NC>(G, V, site_fwd(geo, s, c, mu));
    M3<T> w, r;
    mm<T, 3>(w, gx, u);
    mm_dag<T, 3>(r, w, gf);
    double* d = sm + threadIdx.x * kStagePitch;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      d[2 * q] = (double)r.e[q / 3][q % 3].re;
      d[2 * q + 1] = (double)r.e[q / 3][q % 3].im;
    }
  }
  __syncthreads();
  double2* dst = reinterpret_cast<double2*>(aos + first * 18);
  for (int j = threadIdx.x; j < n * 9; j += blockDim.x) {
    const int m = (2 * j) / 18, k = (2 * j) - m * 18;
    dst[j] = make_double2(sm[m * kStagePitch + k], sm[m * kStagePitch + k + 1]);
  }
}

inline unsigned nblocks(int64_t n, int thr) { return (unsigned)((n + thr - 1) / thr); }

// multiprocessors of the current device (queried once)
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, m = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) ==
                                                   cudaSuccess && m > 0)
      n = m;
    else
      return 1;
  }
  return n;
}

}  // namespace

cudaError_t launch_gradient_grep(int nc, const void* U0, const void* G, void* D, double2* partial, const Geom& geo,
                                 DevState* st, int mode, cudaStream_t s) {
  const double nF = 1.0 / (12.0 * (double)geo.V), nT = 1.0 / (3.0 * (double)geo.V);
  const int64_t full = (geo.V + kGrepThreads - 1) / kGrepThreads;
  const unsigned nb = (unsigned)(full < 2 * sm_count() ? full : 2 * sm_count());
  const auto u = static_cast<const cx<float>*>(U0);
  const auto g = static_cast<const cx<float>*>(G);
  const auto d = static_cast<cx<float>*>(D);
  if (nc == 9)
    return launch_pdl(k_gradient_grep<float, 9>, nb, kGrepThreads, 0, s, u, g, d, partial, geo, st, mode, nF, nT);
  return launch_pdl(k_gradient_grep<float, 6>, nb, kGrepThreads, 0, s, u, g, d, partial, geo, st, mode, nF, nT);
}

template <bool EXACT>
static cudaError_t gstep_launch(int nc, const void* D, void* G, void* g_out, int64_t V, double half_alpha,
                                bool reunit_fp64, const DevState* st, cudaStream_t s) {
  const auto Dp = static_cast<const cx<float>*>(D);
  const auto Gp = static_cast<cx<float>*>(G);
  const auto gp = static_cast<cx<float>*>(g_out);
  const unsigned nb = nblocks(V, 256);
  if (nc == 9) {
    if (reunit_fp64) return launch_pdl(k_gstep<float, 9, double, EXACT>, nb, 256, 0, s, Dp, Gp, gp, V, half_alpha, st);
    return launch_pdl(k_gstep<float, 9, float, EXACT>, nb, 256, 0, s, Dp, Gp, gp, V, half_alpha, st);
  }
  if (reunit_fp64) return launch_pdl(k_gstep<float, 6, double, EXACT>, nb, 256, 0, s, Dp, Gp, gp, V, half_alpha, st);
  return launch_pdl(k_gstep<float, 6, float, EXACT>, nb, 256, 0, s, Dp, Gp, gp, V, half_alpha, st);
}

cudaError_t launch_gstep(int nc, const void* D, void* G, void* g_out, int64_t V, double half_alpha, bool reunit_fp64,
                         bool exact, const DevState* st, cudaStream_t s) {
  if (exact) return gstep_launch<true>(nc, D, G, g_out, V, half_alpha, reunit_fp64, st, s);
  return gstep_launch<false>(nc, D, G, g_out, V, half_alpha, reunit_fp64, st, s);
}

cudaError_t launch_materialize(int nc, const void* U0, const void* G, double* aos, const Geom& geo, cudaStream_t s) {
  const unsigned nb = nblocks(4 * geo.V, kStageMats);
  if (nc == 9)
    k_materialize<float, 9><<<nb, kStageMats, 0, s>>>(static_cast<const cx<float>*>(U0),
                                                       static_cast<const cx<float>*>(G), aos, geo);
  else
    k_materialize<float, 6><<<nb, kStageMats, 0, s>>>(static_cast<const cx<float>*>(U0),
                                                       static_cast<const cx<float>*>(G), aos, geo);
  return cudaPeekAtLastError();
}

}  // namespace lgf
