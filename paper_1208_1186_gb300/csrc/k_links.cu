// Site-local kernels of one gauge-fixing iteration (one thread per lattice
// site, as in the paper's Sec. 2.2, on structure-of-arrays links):
//
//   k_gradient  A(x) = sum_mu [U_mu(x-mu) - U_mu(x)], Delta = A - A^dag -
//               (1/3) Tr(A - A^dag), stored packed as four complex fields
//               (Delta01, Delta02, Delta12, Im Delta00 + i Im Delta11); block
//               partial sums of Re Tr U and Tr Delta Delta^dag in FP64 with
//               warp shuffles.
//               The last block to finish sums the partials in fixed order ->
//               F, theta, and the stop decision of the iteration queue.
//   k_build_g   g(x) = reunitarised (1 + alpha/2 Delta~(x)), or the reunitarised
//               exact exponential exp(alpha/2 Delta~(x)), FP64 arithmetic.
//   k_update    U_mu(x) <- g(x) U_mu(x) g(x+mu)^dag.
//
// Links of direction mu occupy NC complex planes of V elements:
// U[(mu*NC + c)*V + s]; NC = 9 stores every entry, NC = 6 rows 1-2 only.
#include "lgf_df.cuh"
#include "lgf_kernels.cuh"
#include "lgf_reduce.cuh"

namespace lgf {

namespace {

template <class T, int NC>
__device__ __forceinline__ M3<T> load_m3_rw(const cx<T>* base, int64_t V, int64_t s) {
  M3<T> m;
#pragma unroll
  for (int c = 0; c < NC; ++c) m.e[c / 3][c % 3] = base[c * V + s];
  if (NC == 6) complete_row3(m);
  return m;
}

// Gradient of every site, stored packed, and the reduction of F and theta
// (grid_reduce: per-site and per-warp sums in T, FP64 above; the last block
// to arrive adds the block sums in index order, writes F and theta and, in
// mode 1, decides whether this iteration's update is applied).  mode 1
// launches return at once once a previous iteration has stopped the queue.
template <class T, int NC>
__global__ void __launch_bounds__(kGradThreads) k_gradient(const cx<T>* __restrict__ U, cx<T>* __restrict__ D,
                                                           double2* __restrict__ partial, const Geom geo,
                                                           DevState* st, int mode, double normF, double normT) {
  pdl_wait();
  if (queue_stopped(st, mode)) return;
  const int64_t V = geo.V;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T fsum = 0, tsum = 0;
  if (s < V) {
    int c[4];
    site_coords(geo, s, c);
    M3<T> A;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A.e[i][j] = mk<T>(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const cx<T>* base = U + (int64_t)mu * NC * V;
      const M3<T> own = load_m3<T, NC>(base, V, s);
      const M3<T> back = load_m3<T, NC>(base, V, site_back(geo, s, c, mu));
      fsum += own.e[0][0].re + own.e[1][1].re + own.e[2][2].re;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A.e[i][j] = A.e[i][j] + (back.e[i][j] - own.e[i][j]);
    }
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
    tsum = 2 * (norm2(d01) + norm2(d02) + norm2(d12)) + i0 * i0 + i1 * i1 + i2 * i2;
  }
  grid_reduce<T>(fsum, tsum, partial, st, normF, normT, mode);
}

template <class T, int NC, class RT, bool EXACT>
__global__ void __launch_bounds__(256) k_build_g(const cx<T>* __restrict__ D, cx<T>* __restrict__ g, int64_t V,
                                                 double hd, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const RT h = (RT)hd;
  const cx<RT> c0 = cvt<RT>(ldg(D + s));
  const cx<RT> c1 = cvt<RT>(ldg(D + V + s));
  const cx<RT> c2 = cvt<RT>(ldg(D + 2 * V + s));
  const cx<RT> c3 = cvt<RT>(ldg(D + 3 * V + s));
  M3<RT> m;
  if constexpr (EXACT) {  // the exact exponential of h Delta~ (expm_taylor)
    m = expm_taylor(unpack_ah(c0, c1, c2, c3, h));
  } else {
    // rows 1-2 of 1 + h Delta~; Delta~10 = -conj(Delta~01), Delta~_ii = i Im
    m.e[0][0] = mk<RT>(1, h * c3.re);
    m.e[0][1] = scale(c0, h);
    m.e[0][2] = scale(c1, h);
    m.e[1][0] = mk<RT>(-h * c0.re, h * c0.im);
    m.e[1][1] = mk<RT>(1, h * c3.im);
    m.e[1][2] = scale(c2, h);
  }
  reunitarize(m);
#pragma unroll
  for (int c = 0; c < NC; ++c) g[c * V + s] = cvt<T>(m.e[c / 3][c % 3]);
}

template <class T, int NC>
__global__ void __launch_bounds__(256) k_update(cx<T>* U, const cx<T>* __restrict__ g, const Geom geo,
                                                const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int64_t V = geo.V;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(geo, s, c);
  const M3<T> gx = load_m3<T, NC>(g, V, s);
  constexpr int ROWS = NC / 3;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    cx<T>* base = U + (int64_t)mu * NC * V;
    const M3<T> u = load_m3_rw<T, NC>(base, V, s);
    const M3<T> gf = load_m3<T, NC>(g, V, site_fwd(geo, s, c, mu));
    M3<T> w, r;
    mm<T, ROWS>(w, gx, u);
    mm_dag<T, ROWS>(r, w, gf);
#pragma unroll
    for (int q = 0; q < NC; ++q) base[q * V + s] = r.e[q / 3][q % 3];
  }
}

// one thread per (site, matrix): 18 doubles in, NC complex out; nmu matrices
// per site (4 for links, 1 for a gauge field)
template <class T, int NC>
__global__ void k_aos_to_soa(const double* __restrict__ aos, cx<T>* __restrict__ U, int64_t V, int nmu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nmu * V) return;
  const int64_t s = i / nmu;
  const int mu = (int)(i - s * nmu);
  const double* src = aos + i * 18;
#pragma unroll
  for (int c = 0; c < NC; ++c) U[((int64_t)mu * NC + c) * V + s] = mk<T>((T)src[2 * c], (T)src[2 * c + 1]);
}

// ---------------------------------------------------------------------------
// Link loads and stores in the host layout (AoS, 18 doubles per link, 4 links
// per site), staged through shared memory.  A CTA moves one contiguous chunk
// of kStageMats links with 16-byte accesses; the staged rows have a pitch of
// 19 doubles, which makes the per-thread 8-byte reads conflict-free.  The AoS
// side may be host memory that the device reads or writes directly (pinned
// memory over NVLink-C2C): every byte crosses once, coalesced.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stage_in(const double* __restrict__ aos, double* sm, int64_t first, int n) {
  const double2* src = reinterpret_cast<const double2*>(aos + first * 18);
  for (int j = threadIdx.x; j < n * 9; j += blockDim.x) {
    const double2 v = src[j];  // doubles 2j and 2j+1 of the chunk: one link, entries k and k+1
    const int m = (2 * j) / 18, k = (2 * j) - m * 18;
    sm[m * kStagePitch + k] = v.x;
    sm[m * kStagePitch + k + 1] = v.y;
  }
}

__device__ __forceinline__ void stage_out(const double* sm, double* __restrict__ aos, int64_t first, int n) {
  double2* dst = reinterpret_cast<double2*>(aos + first * 18);
  for (int j = threadIdx.x; j < n * 9; j += blockDim.x) {
    const int m = (2 * j) / 18, k = (2 * j) - m * 18;
    dst[j] = make_double2(sm[m * kStagePitch + k], sm[m * kStagePitch + k + 1]);
  }
}

// AoS links -> FP64 SoA (NC64 planes per direction, 0: none) and FP32 SoA
// (NC32 planes, 0: none), one read of the input
template <int NC64, int NC32>
__global__ void __launch_bounds__(kStageMats) k_load_aos(const double* __restrict__ aos, cx<double>* __restrict__ U64,
                                                         cx<float>* __restrict__ U32, int64_t V) {
  __shared__ double sm[kStageMats * kStagePitch];
  const int64_t first = (int64_t)blockIdx.x * kStageMats;
  const int n = (int)(4 * V - first < kStageMats ? 4 * V - first : kStageMats);
  stage_in(aos, sm, first, n);
  __syncthreads();
  if ((int)threadIdx.x >= n) return;
  const int64_t i = first + threadIdx.x;
  const int64_t s = i >> 2;
  const int mu = (int)(i & 3);
  const double* m = sm + threadIdx.x * kStagePitch;
#pragma unroll
  for (int c = 0; c < NC64; ++c) U64[((int64_t)mu * NC64 + c) * V + s] = mk<double>(m[2 * c], m[2 * c + 1]);
#pragma unroll
  for (int c = 0; c < NC32; ++c)
    U32[((int64_t)mu * NC32 + c) * V + s] = mk<float>((float)m[2 * c], (float)m[2 * c + 1]);
}

// SoA links (rows 1-2 rebuilt for NC = 6) -> AoS doubles
template <class T, int NC>
__global__ void __launch_bounds__(kStageMats) k_store_aos(const cx<T>* __restrict__ U, double* __restrict__ aos,
                                                          int64_t V) {
  __shared__ double sm[kStageMats * kStagePitch];
  const int64_t first = (int64_t)blockIdx.x * kStageMats;
  const int n = (int)(4 * V - first < kStageMats ? 4 * V - first : kStageMats);
  if ((int)threadIdx.x < n) {
    const int64_t i = first + threadIdx.x;
    const int64_t s = i >> 2;
    const int mu = (int)(i & 3);
    const M3<T> m = load_m3<T, NC>(U + (int64_t)mu * NC * V, V, s);
    double* d = sm + threadIdx.x * kStagePitch;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      d[2 * c] = (double)m.e[c / 3][c % 3].re;
      d[2 * c + 1] = (double)m.e[c / 3][c % 3].im;
    }
  }
  __syncthreads();
  stage_out(sm, aos, first, n);
}

// double-float links (36 hi planes, then 36 lo planes) -> AoS doubles, each
// entry hi + lo; with eta (not null: hi planes, then lo planes) the links
// (1 + eta(x)) U (1 + eta(x+mu))^dag of the tail's gauge representation,
// formed in double-float
__global__ void __launch_bounds__(kStageMats) k_store_aos_df(const cx<float>* __restrict__ Uh,
                                                             const cx<float>* __restrict__ Ul,
                                                             const cx<float>* __restrict__ eta, const Geom geo,
                                                             double* __restrict__ aos) {
  __shared__ double sm[kStageMats * kStagePitch];
  const int V = (int)geo.V;
  const int64_t first = (int64_t)blockIdx.x * kStageMats;
  const int n = (int)(4 * (int64_t)V - first < kStageMats ? 4 * (int64_t)V - first : kStageMats);
  if ((int)threadIdx.x < n) {
    const int64_t i = first + threadIdx.x;
    const int s = (int)(i >> 2);
    const int mu = (int)(i & 3);
    M3<float> uh;
    cx<float> ul[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const int o = (mu * 9 + c) * V + s;
      uh.e[c / 3][c % 3] = ldg(Uh + o);
      ul[c] = ldg(Ul + o);
    }
    df re[9], im[9];
    if (eta != nullptr) {
      int x[4];
      site_coords_i(geo.L, s, x);
      const int cm = mu == 0 ? x[0] : mu == 1 ? x[1] : mu == 2 ? x[2] : x[3];
      const int Lm = mu == 0 ? geo.L[0] : mu == 1 ? geo.L[1] : mu == 2 ? geo.L[2] : geo.L[3];
      const int st = mu == 0 ? 1 : mu == 1 ? geo.L[0] : mu == 2 ? geo.L[0] * geo.L[1] : geo.L[0] * geo.L[1] * geo.L[2];
      const int sf = cm < Lm - 1 ? s + st : s - (Lm - 1) * st;
      const cx<float>* el = eta + 9 * V;
      const M3<float> xh = load_m3i<float, 9>(eta, V, s), xl = load_m3i<float, 9>(el, V, s);
      const M3<float> fh = load_m3i<float, 9>(eta, V, sf), fl = load_m3i<float, 9>(el, V, sf);
      tail_link_exact(uh, ul, xh, xl, fh, fl, re, im);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        re[c] = {uh.e[c / 3][c % 3].re, ul[c].re};
        im[c] = {uh.e[c / 3][c % 3].im, ul[c].im};
      }
    }
    double* d = sm + threadIdx.x * kStagePitch;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      d[2 * c] = df_to_double(re[c].h, re[c].l);
      d[2 * c + 1] = df_to_double(im[c].h, im[c].l);
    }
  }
  __syncthreads();
  stage_out(sm, aos, first, n);
}

template <class T, int NC>
__global__ void k_soa_to_aos(const cx<T>* __restrict__ U, double* __restrict__ aos, int64_t V, int nmu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nmu * V) return;
  const int64_t s = i / nmu;
  const int mu = (int)(i - s * nmu);
  const M3<T> m = load_m3<T, NC>(U + (int64_t)mu * NC * V, V, s);
  double* dst = aos + i * 18;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    dst[2 * c] = (double)m.e[c / 3][c % 3].re;
    dst[2 * c + 1] = (double)m.e[c / 3][c % 3].im;
  }
}

// G(x) <- reunitarised g(x) G(x), in the storage precision
template <class T, int NC>
__global__ void __launch_bounds__(256) k_accumulate(cx<T>* G, const cx<T>* __restrict__ g, int64_t V,
                                                    const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const M3<T> a = load_m3<T, NC>(g, V, s);
  const M3<T> b = load_m3_rw<T, NC>(G, V, s);
  M3<T> r;
  mm<T, 2>(r, a, b);
  reunitarize(r);
#pragma unroll
  for (int c = 0; c < NC; ++c) G[c * V + s] = r.e[c / 3][c % 3];
}

// FP64 copy of a stored gauge field, reunitarised in FP64: out has 9 planes
template <class T, int NC>
__global__ void __launch_bounds__(256) k_promote_gauge(const cx<T>* __restrict__ G, cx<double>* __restrict__ out,
                                                       int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const M3<T> a = load_m3<T, NC>(G, V, s);
  M3<double> m;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m.e[i][j] = cvt<double>(a.e[i][j]);
  reunitarize(m);
#pragma unroll
  for (int c = 0; c < 9; ++c) out[c * V + s] = m.e[c / 3][c % 3];
}

template <class T, int NC>
__global__ void k_set_identity(cx<T>* __restrict__ G, int64_t V) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) G[c * V + s] = mk<T>((c % 4 == 0) ? (T)1 : (T)0, (T)0);
}

template <class T>
__global__ void k_unpack_fields(const cx<T>* __restrict__ D, double* __restrict__ out, int64_t V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * V) return;
  const int64_t s = i >> 2;
  const int f = (int)(i & 3);
  const cx<T> v = D[(int64_t)f * V + s];
  out[2 * i] = (double)v.re;
  out[2 * i + 1] = (double)v.im;
}

inline unsigned blocks_for(int64_t n, int thr) { return (unsigned)((n + thr - 1) / thr); }

}  // namespace

#define LGF_DISPATCH(prec, nc, KERNEL_CALL)         \
  do {                                              \
    if ((prec) == 8 && (nc) == 9) {                 \
      using T = double;                             \
      constexpr int NC = 9;                         \
      KERNEL_CALL;                                  \
    } else if ((prec) == 8) {                       \
      using T = double;                             \
      constexpr int NC = 6;                         \
      KERNEL_CALL;                                  \
    } else if ((nc) == 9) {                         \
      using T = float;                              \
      constexpr int NC = 9;                         \
      KERNEL_CALL;                                  \
    } else {                                        \
      using T = float;                              \
      constexpr int NC = 6;                         \
      KERNEL_CALL;                                  \
    }                                               \
  } while (0)

cudaError_t launch_gradient(int prec, int nc, const void* U, void* D, double2* partial, const Geom& geo,
                            DevState* st, int mode, cudaStream_t s) {
  const unsigned nb = (unsigned)gradient_blocks(geo.V);
  const double nF = 1.0 / (12.0 * (double)geo.V), nT = 1.0 / (3.0 * (double)geo.V);
  LGF_DISPATCH(prec, nc,
               (launch_pdl(k_gradient<T, NC>, nb, kGradThreads, 0, s, static_cast<const cx<T>*>(U),
                           static_cast<cx<T>*>(D), partial, geo, st, mode, nF, nT)));
  return cudaPeekAtLastError();
}

template <bool EXACT>
static cudaError_t build_g_launch(int prec, int nc, const void* D, void* g, int64_t V, double half_alpha,
                                  bool reunit_fp64, const DevState* st, cudaStream_t s) {
  if (prec == 4 && !reunit_fp64) {
    if (nc == 9)
      launch_pdl(k_build_g<float, 9, float, EXACT>, blocks_for(V, 256), 256, 0, s, static_cast<const cx<float>*>(D),
                 static_cast<cx<float>*>(g), V, half_alpha, st);
    else
      launch_pdl(k_build_g<float, 6, float, EXACT>, blocks_for(V, 256), 256, 0, s, static_cast<const cx<float>*>(D),
                 static_cast<cx<float>*>(g), V, half_alpha, st);
    return cudaPeekAtLastError();
  }
  LGF_DISPATCH(prec, nc,
               (launch_pdl(k_build_g<T, NC, double, EXACT>, blocks_for(V, 256), 256, 0, s,
                           static_cast<const cx<T>*>(D), static_cast<cx<T>*>(g), V, half_alpha, st)));
  return cudaPeekAtLastError();
}

cudaError_t launch_build_g(int prec, int nc, const void* D, void* g, int64_t V, double half_alpha,
                           bool reunit_fp64, bool exact, const DevState* st, cudaStream_t s) {
  if (exact) return build_g_launch<true>(prec, nc, D, g, V, half_alpha, reunit_fp64, st, s);
  return build_g_launch<false>(prec, nc, D, g, V, half_alpha, reunit_fp64, st, s);
}

cudaError_t launch_update(int prec, int nc, void* U, const void* g, const Geom& geo, const DevState* st,
                          cudaStream_t s) {
  LGF_DISPATCH(prec, nc,
               (launch_pdl(k_update<T, NC>, blocks_for(geo.V, 256), 256, 0, s, static_cast<cx<T>*>(U),
                                                                       static_cast<const cx<T>*>(g), geo, st)));
  return cudaPeekAtLastError();
}

cudaError_t launch_aos_to_soa(int prec, int nc, const double* aos, void* U, int64_t V, int nmu, cudaStream_t s) {
  LGF_DISPATCH(prec, nc,
               (k_aos_to_soa<T, NC><<<blocks_for(nmu * V, 256), 256, 0, s>>>(aos, static_cast<cx<T>*>(U), V, nmu)));
  return cudaPeekAtLastError();
}

cudaError_t launch_load_aos(int nc64, int nc32, const double* aos, void* U64, void* U32, int64_t V, cudaStream_t s) {
  const unsigned nb = blocks_for(4 * V, kStageMats);
  auto d = static_cast<cx<double>*>(U64);
  auto f = static_cast<cx<float>*>(U32);
  if (nc64 == 9 && nc32 == 9) k_load_aos<9, 9><<<nb, kStageMats, 0, s>>>(aos, d, f, V);
  else if (nc64 == 9 && nc32 == 6) k_load_aos<9, 6><<<nb, kStageMats, 0, s>>>(aos, d, f, V);
  else if (nc64 == 9 && nc32 == 0) k_load_aos<9, 0><<<nb, kStageMats, 0, s>>>(aos, d, f, V);
  else if (nc64 == 6 && nc32 == 0) k_load_aos<6, 0><<<nb, kStageMats, 0, s>>>(aos, d, f, V);
  else return cudaErrorInvalidValue;
  return cudaPeekAtLastError();
}

cudaError_t launch_store_aos(int prec, int nc, const void* U, double* aos, int64_t V, cudaStream_t s) {
  const unsigned nb = blocks_for(4 * V, kStageMats);
  LGF_DISPATCH(prec, nc, (k_store_aos<T, NC><<<nb, kStageMats, 0, s>>>(static_cast<const cx<T>*>(U), aos, V)));
  return cudaPeekAtLastError();
}

cudaError_t launch_soa_to_aos(int prec, int nc, const void* U, double* aos, int64_t V, int nmu, cudaStream_t s) {
  LGF_DISPATCH(prec, nc,
               (k_soa_to_aos<T, NC><<<blocks_for(nmu * V, 256), 256, 0, s>>>(static_cast<const cx<T>*>(U), aos, V,
                                                                             nmu)));
  return cudaPeekAtLastError();
}

cudaError_t launch_accumulate(int prec, int nc, void* G, const void* g, int64_t V, const DevState* st,
                              cudaStream_t s) {
  LGF_DISPATCH(prec, nc,
               (launch_pdl(k_accumulate<T, NC>, blocks_for(V, 256), 256, 0, s, static_cast<cx<T>*>(G),
                                                                       static_cast<const cx<T>*>(g), V, st)));
  return cudaPeekAtLastError();
}

cudaError_t launch_promote_gauge(int prec, int nc, const void* G, void* out64, int64_t V, cudaStream_t s) {
  LGF_DISPATCH(prec, nc,
               (k_promote_gauge<T, NC><<<blocks_for(V, 256), 256, 0, s>>>(static_cast<const cx<T>*>(G),
                                                                          static_cast<cx<double>*>(out64), V)));
  return cudaPeekAtLastError();
}

cudaError_t launch_store_aos_df(const void* Udf, const void* eta, const Geom& geo, double* aos, cudaStream_t s) {
  auto h = static_cast<const cx<float>*>(Udf);
  k_store_aos_df<<<blocks_for(4 * geo.V, kStageMats), kStageMats, 0, s>>>(h, h + 36 * geo.V,
                                                                          static_cast<const cx<float>*>(eta), geo, aos);
  return cudaPeekAtLastError();
}

cudaError_t launch_set_identity(int prec, int nc, void* G, int64_t V, cudaStream_t s) {
  LGF_DISPATCH(prec, nc, (k_set_identity<T, NC><<<blocks_for(V, 256), 256, 0, s>>>(static_cast<cx<T>*>(G), V)));
  return cudaPeekAtLastError();
}

cudaError_t launch_unpack_fields(int prec, const void* D, double* out, int64_t V, cudaStream_t s) {
  if (prec == 8)
    k_unpack_fields<double><<<blocks_for(4 * V, 256), 256, 0, s>>>(static_cast<const cx<double>*>(D), out, V);
  else
    k_unpack_fields<float><<<blocks_for(4 * V, 256), 256, 0, s>>>(static_cast<const cx<float>*>(D), out, V);
  return cudaPeekAtLastError();
}

}  // namespace lgf
