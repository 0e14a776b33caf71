// Fourier acceleration on chip: the 4D transform of the packed gradient is
// done as an x-y plane transform and a z-t plane transform (the paper's
// "2D plus 2D" split, Sec. 2.2), each staged in shared memory with a
// mixed-radix Stockham FFT (radices 4, 2, 3, 5).
//
//   k_fft_xy : one CTA per (z, t) plane and field; forward or inverse
//              transform along x then y.
//   k_fft_zt : one CTA per (y, run of Bx consecutive x); for each of the four
//              fields: forward transform along z and t, multiplication by
//              p2_max / (V p2(k)) (0 at k = 0), inverse transform along t
//              and z.  The forward x-y pass runs before it and the inverse
//              x-y pass after it, so the data crosses HBM three times.
//
// Stockham stage (Govindaraju et al., SC'08 formulation): with Ns the
// product of the radices already applied, butterfly j of a line reads
// in[j + r*L/R], multiplies input r by W_L^(r * (j mod Ns) * L/(Ns R)), does
// an R-point DFT and writes out[(j / Ns) Ns R + (j mod Ns) + r Ns].
#include "lgf_kernels.cuh"

namespace lgf {

namespace {

// R-point DFT in registers; forward uses e^{-2 pi i/R}, inverse e^{+2 pi i/R}.
template <class T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a, bool neg) {  // neg ? -i*a : +i*a
  return neg ? mk<T>(a.im, -a.re) : mk<T>(-a.im, a.re);
}

template <class T, int R>
struct Butterfly;

template <class T>
struct Butterfly<T, 2> {
  __device__ __forceinline__ static void run(cx<T>* v, bool) {
    cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <class T>
struct Butterfly<T, 4> {
  __device__ __forceinline__ static void run(cx<T>* v, bool inv) {
    cx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
    cx<T> s13 = v[1] + v[3], d13 = mul_i(v[1] - v[3], !inv);  // -i (fwd) / +i (inv)
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = d02 + d13;
    v[3] = d02 - d13;
  }
};

template <class T>
struct Butterfly<T, 3> {
  __device__ __forceinline__ static void run(cx<T>* v, bool inv) {
    const T h = (T)0.5;
    const T s = (T)0.86602540378443864676;  // sin(2 pi / 3)
    cx<T> t1 = v[1] + v[2];
    cx<T> t2 = scale(mul_i(v[1] - v[2], !inv), s);  // -i s (v1 - v2) forward
    cx<T> m = v[0] - scale(t1, h);
    v[0] = v[0] + t1;
    v[1] = m + t2;
    v[2] = m - t2;
  }
};

template <class T>
struct Butterfly<T, 5> {
  __device__ __forceinline__ static void run(cx<T>* v, bool inv) {
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
    const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
    cx<T> a1 = v[1] + v[4], b1 = v[1] - v[4];
    cx<T> a2 = v[2] + v[3], b2 = v[2] - v[3];
    cx<T> p1 = v[0] + scale(a1, c1) + scale(a2, c2);
    cx<T> p2 = v[0] + scale(a1, c2) + scale(a2, c1);
    cx<T> q1 = mul_i(scale(b1, s1) + scale(b2, s2), !inv);  // -i(...) forward
    cx<T> q2 = mul_i(scale(b1, s2) - scale(b2, s1), !inv);
    v[0] = v[0] + a1 + a2;
    v[1] = p1 + q1;
    v[4] = p1 - q1;
    v[2] = p2 + q2;
    v[3] = p2 - q2;
  }
};

// A batch of lines in shared memory: line l starts at
// (l % na) * sa + (l / na) * sb and its elements are es apart.
struct Lines {
  int n, na, sa, sb, es;
  __device__ __forceinline__ int offset(int l) const { return (l % na) * sa + (l / na) * sb; }
};

template <class T, int R>
__device__ __forceinline__ void stockham_stage(const cx<T>* __restrict__ in, cx<T>* __restrict__ out,
                                               int L, int Ns, const Lines& ln,
                                               const cx<T>* __restrict__ tw, bool inv) {
  const int nb = L / R;
  const int total = nb * ln.n;
  const int twstep = L / (Ns * R);
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int line = w % ln.n;
    const int j = w / ln.n;
    const int base = ln.offset(line);
    const int k = j % Ns;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[base + (j + r * nb) * ln.es];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = v[r] * tw[r * k * twstep];
    Butterfly<T, R>::run(v, inv);
    const int d = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[base + (d + r * Ns) * ln.es] = v[r];
  }
}

// Transform every line of `ln` along one axis; the result ends in `cur`.
template <class T>
__device__ void fft_lines(cx<T>*& cur, cx<T>*& oth, const AxisPlan& ap, const Lines& ln,
                          const cx<T>* tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < ap.nst; ++s) {
    const int R = ap.radix[s];
    switch (R) {
      case 4: stockham_stage<T, 4>(cur, oth, ap.L, Ns, ln, tw, inv); break;
      case 2: stockham_stage<T, 2>(cur, oth, ap.L, Ns, ln, tw, inv); break;
      case 3: stockham_stage<T, 3>(cur, oth, ap.L, Ns, ln, tw, inv); break;
      default: stockham_stage<T, 5>(cur, oth, ap.L, Ns, ln, tw, inv); break;
    }
    __syncthreads();
    cx<T>* t = cur;
    cur = oth;
    oth = t;
    Ns *= R;
  }
}

template <class T>
__device__ __forceinline__ void load_twiddles(cx<T>* dst, const cx<T>* __restrict__ src, int L, bool inv) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    cx<T> w = src[i];
    dst[i] = inv ? conj(w) : w;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_fft_xy(cx<T>* __restrict__ D, const __grid_constant__ FftGeom fg,
                                                const cx<T>* __restrict__ tw, int inverse,
                                                const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Lx = fg.L[0], Ly = fg.L[1];
  const int P = fg.Pxy;
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + P * Ly;
  cx<T>* twx = buf1 + P * Ly;
  cx<T>* twy = twx + kMaxL;
  const bool inv = inverse != 0;
  load_twiddles(twx, tw + 0 * kMaxL, Lx, inv);
  load_twiddles(twy, tw + 1 * kMaxL, Ly, inv);
  const int64_t base = (int64_t)blockIdx.y * fg.V + (int64_t)blockIdx.x * (Lx * Ly);
  const int n = Lx * Ly;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int x = i % Lx, y = i / Lx;
    buf0[y * P + x] = D[base + i];
  }
  __syncthreads();
  cx<T>* cur = buf0;
  cx<T>* oth = buf1;
  const Lines xl{Ly, Ly, P, 0, 1};  // lines y, contiguous along x
  fft_lines(cur, oth, fg.ax[0], xl, twx, inv);
  const Lines yl{Lx, Lx, 1, 0, P};  // lines x, stride P along y
  fft_lines(cur, oth, fg.ax[1], yl, twy, inv);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int x = i % Lx, y = i / Lx;
    D[base + i] = cur[y * P + x];
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_fft_zt(cx<T>* __restrict__ D, const __grid_constant__ FftGeom fg,
                                                const cx<T>* __restrict__ tw,
                                                const double* __restrict__ sin2,
                                                const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Lx = fg.L[0], Ly = fg.L[1], Lz = fg.L[2], Lt = fg.L[3];
  const int Bx = fg.Bx, Pt = fg.Pt;
  const int tile = Pt * Lt;
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + tile;
  cx<T>* twz = buf1 + tile;
  cx<T>* twt = twz + kMaxL;
  cx<T>* twzi = twt + kMaxL;
  cx<T>* twti = twzi + kMaxL;
  T* kfac = reinterpret_cast<T*>(twti + kMaxL);
  load_twiddles(twz, tw + 2 * kMaxL, Lz, false);
  load_twiddles(twt, tw + 3 * kMaxL, Lt, false);
  load_twiddles(twzi, tw + 2 * kMaxL, Lz, true);
  load_twiddles(twti, tw + 3 * kMaxL, Lt, true);

  const int nxc = Lx / Bx;
  const int x0 = (blockIdx.x % nxc) * Bx;
  const int y = blockIdx.x / nxc;
  const int n = Bx * Lz * Lt;
  // acceleration factor p2_max / (V p2(k)) of every point of the tile
  {
    const double sxy_base = sin2[1 * kMaxL + y];
    const double invV = 1.0 / (double)fg.V;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int xb = i % Bx, q = i / Bx, z = q % Lz, t = q / Lz;
      const int kx = x0 + xb;
      double f = 0.0;
      if ((kx | y | z | t) != 0) {
        const double p2 = sin2[kx] + sxy_base + sin2[2 * kMaxL + z] + sin2[3 * kMaxL + t];
        f = fg.p2max / p2 * invV;
      }
      kfac[xb + Bx * z + Pt * t] = (T)f;
    }
  }
  const int64_t col = x0 + (int64_t)Lx * y;
  const int64_t zstride = (int64_t)Lx * Ly;
  const Lines zl{Bx * Lt, Bx, 1, Pt, Bx};  // lines (xb, t), stride Bx along z
  const Lines tl{Bx * Lz, Bx * Lz, 1, 0, Pt};  // lines (xb, z), stride Pt along t
  for (int f = 0; f < 4; ++f) {
    cx<T>* Df = D + (int64_t)f * fg.V + col;
    cx<T>* cur = buf0;
    cx<T>* oth = buf1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int xb = i % Bx, q = i / Bx, z = q % Lz, t = q / Lz;
      cur[xb + Bx * z + Pt * t] = Df[xb + zstride * (z + (int64_t)Lz * t)];
    }
    __syncthreads();
    fft_lines(cur, oth, fg.ax[2], zl, twz, false);
    fft_lines(cur, oth, fg.ax[3], tl, twt, false);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int xb = i % Bx, q = i / Bx, z = q % Lz, t = q / Lz;
      const int a = xb + Bx * z + Pt * t;
      cur[a] = scale(cur[a], kfac[a]);
    }
    __syncthreads();
    fft_lines(cur, oth, fg.ax[3], tl, twti, true);
    fft_lines(cur, oth, fg.ax[2], zl, twzi, true);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int xb = i % Bx, q = i / Bx, z = q % Lz, t = q / Lz;
      Df[xb + zstride * (z + (int64_t)Lz * t)] = cur[xb + Bx * z + Pt * t];
    }
    __syncthreads();
  }
}

}  // namespace

bool make_axis_plan(int L, AxisPlan* p) {
  if (L < 2 || L > kMaxL) return false;
  p->L = L;
  p->nst = 0;
  int n = L;
  while (n % 4 == 0 && p->nst < kMaxStages) {
    p->radix[p->nst++] = 4;
    n /= 4;
  }
  const int rest[3] = {2, 3, 5};
  for (int r : rest)
    while (n % r == 0 && p->nst < kMaxStages) {
      p->radix[p->nst++] = r;
      n /= r;
    }
  return n == 1;
}

size_t fft_xy_smem(const FftGeom& fg, int real_bytes) {
  const size_t c = 2 * (size_t)real_bytes;
  return (2 * (size_t)fg.Pxy * fg.L[1] + 2 * kMaxL) * c;
}

size_t fft_zt_smem(const FftGeom& fg, int real_bytes) {
  const size_t c = 2 * (size_t)real_bytes;
  const size_t tile = (size_t)fg.Pt * fg.L[3];
  return (2 * tile + 4 * kMaxL) * c + tile * real_bytes;
}

cudaError_t fft_set_smem_limits(int real_bytes, size_t xy, size_t zt) {
  cudaError_t e;
  if (real_bytes == 8) {
    e = cudaFuncSetAttribute(k_fft_xy<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xy);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fft_zt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zt);
  }
  e = cudaFuncSetAttribute(k_fft_xy<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xy);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fft_zt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zt);
}

static int fft_threads(int points) {
  int t = (points / 4 + 31) / 32 * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}

cudaError_t launch_fft_xy(int prec, void* D, const FftGeom& fg, const void* tw, int inverse,
                          const DevState* st, cudaStream_t s) {
  dim3 grid(fg.L[2] * fg.L[3], 4);
  const int thr = fft_threads(fg.L[0] * fg.L[1]);
  if (prec == 8) {
    launch_pdl(k_fft_xy<double>, grid, thr, fft_xy_smem(fg, 8), s, static_cast<cx<double>*>(D), fg,
                                                           static_cast<const cx<double>*>(tw), inverse, st);
  } else {
    launch_pdl(k_fft_xy<float>, grid, thr, fft_xy_smem(fg, 4), s, static_cast<cx<float>*>(D), fg,
                                                          static_cast<const cx<float>*>(tw), inverse, st);
  }
  return cudaPeekAtLastError();
}

cudaError_t launch_fft_zt(int prec, void* D, const FftGeom& fg, const void* tw, const double* sin2,
                          const DevState* st, cudaStream_t s) {
  dim3 grid((fg.L[0] / fg.Bx) * fg.L[1]);
  const int thr = fft_threads(fg.Bx * fg.L[2] * fg.L[3]);
  if (prec == 8) {
    launch_pdl(k_fft_zt<double>, grid, thr, fft_zt_smem(fg, 8), s, static_cast<cx<double>*>(D), fg,
                                                           static_cast<const cx<double>*>(tw), sin2, st);
  } else {
    launch_pdl(k_fft_zt<float>, grid, thr, fft_zt_smem(fg, 4), s, static_cast<cx<float>*>(D), fg,
                                                          static_cast<const cx<float>*>(tw), sin2, st);
  }
  return cudaPeekAtLastError();
}

}  // namespace lgf
