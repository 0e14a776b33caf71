// Fourier acceleration as one-axis passes with in-register line FFTs
// (fft_reg.cuh).  The packed gradient D[f][s] (four complex fields) is
// transformed in place:
//
//   xpass(fwd) -> strided(y, fwd) -> strided(z, fwd) -> tpass -> strided(z, inv)
//   -> strided(y, inv) -> xpass(inv)
//
// tpass does the forward t transform, multiplies by the acceleration factor
// p2_max / (V p2(k)) (0 at k = 0; tabulated per site in the digit-reversed
// order the forward passes leave) and the inverse t transform, all in
// registers.  The paper (Sec. 2.2) splits its 4D FFT into 2D plus 2D library
// transforms; here each pass streams the 4 fields once with every line in
// one thread's registers, so the index arithmetic and twiddles fold into
// constants.
//
// Coalescing: in the strided passes consecutive threads own lines at
// consecutive x, so every load and store of a warp covers 32 consecutive
// complex numbers.  x-lines are contiguous, so xpass stages a tile of lines
// through shared memory (row pitch L + 1: conflict-free row reads).
#include "fft_reg.cuh"
#include "lgf_kernels.cuh"

namespace lgf {

namespace {

template <class T, int L>
constexpr int xpass_lines() {
  return (L * (int)sizeof(cx<T>) > 256) ? 64 : 128;
}

// One thread per x-line; the block's lines are a contiguous chunk of D.
template <class T, int L, bool INV>
__global__ void __launch_bounds__(128) k_xpass(cx<T>* __restrict__ D, int64_t total_lines,
                                               const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int NL = xpass_lines<T, L>();
  constexpr int P = L + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw);
  const int64_t g0 = (int64_t)blockIdx.x * NL;
  const int nl = (int)((total_lines - g0) < NL ? (total_lines - g0) : NL);
  cx<T>* chunk = D + g0 * L;
  const int ne = nl * L;
  constexpr int PER = NL * L / 128;  // elements per thread of a full tile
  if (nl == NL) {  // full tile: every load of a thread in flight at once
    cx<T> r[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) r[k] = chunk[threadIdx.x + 128 * k];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + 128 * k;
      tile[(e / L) * P + (e % L)] = r[k];
    }
  } else {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) tile[(e / L) * P + (e % L)] = chunk[e];
  }
  __syncthreads();
  for (int ln = threadIdx.x; ln < nl; ln += blockDim.x) {
    cx<T> v[L];
    cx<T>* row = tile + ln * P;
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = row[p];
    if (INV)
      regfft::inverse<T, L>(v);
    else
      regfft::forward<T, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) row[p] = v[p];
  }
  __syncthreads();
  if (nl == NL) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + 128 * k;
      chunk[e] = tile[(e / L) * P + (e % L)];
    }
  } else {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) chunk[e] = tile[(e / L) * P + (e % L)];
  }
}

// One thread per line along an axis of stride S (y: Lx, z: Lx*Ly).
// FP32 lines up to 32 points: four 128-thread blocks per SM (128 registers)
template <class T, int L>
constexpr int pass_min_blocks() {
  return (sizeof(T) == 4 && L <= 32) ? 4 : 1;
}

template <class T, int L, bool INV>
__global__ void __launch_bounds__(128, pass_min_blocks<T, L>()) k_strided(cx<T>* __restrict__ D, int64_t V, int64_t S,
                                                 const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  // 32-bit offsets: 4 V < 2^31 for extents <= 64
  const int nl = (int)(V / L);  // lines per field
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 4 * nl) return;
  const int Si = (int)S;
  const int f = g / nl, l = g - f * nl;
  cx<T>* line = D + (f * (int)V + (l % Si) + (l / Si) * Si * L);
  cx<T> v[L];
#pragma unroll
  for (int p = 0; p < L; ++p) v[p] = line[p * Si];
  if (INV)
    regfft::inverse<T, L>(v);
  else
    regfft::forward<T, L>(v);
#pragma unroll
  for (int p = 0; p < L; ++p) line[p * Si] = v[p];
}

// One thread per t-line: forward t, times the acceleration factor, inverse t.
// FP64 reads the factor from the per-site table kfac (an FP64 division per
// mode would be slow on this GPU); FP32 forms it from the per-axis tables
// s2p[axis][position] = 4 sin^2(pi k / L) at the digit-reversed frequency k
// of each position: K = p2max / V / (s2x + s2y + s2z + s2t), 0 at k = 0.
template <class T, int L>
__global__ void __launch_bounds__(128, pass_min_blocks<T, L>()) k_tpass(cx<T>* __restrict__ D, int64_t V, int Lx, int Ly,
                                               const T* __restrict__ kfac, const float* __restrict__ s2p,
                                               float c_over_V, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  __shared__ float s2t[kMaxL];
  if (sizeof(T) == 4)
    for (int i = threadIdx.x; i < L; i += blockDim.x) s2t[i] = s2p[3 * kMaxL + i];
  __syncthreads();
  const int S = (int)(V / L);  // 32-bit offsets: 4 V < 2^31 for extents <= 64
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 4 * S) return;
  const int f = g / S, l = g - f * S;
  cx<T>* line = D + (f * (int)V + l);
  cx<T> v[L];
#pragma unroll
  for (int p = 0; p < L; ++p) v[p] = line[p * S];
  regfft::forward<T, L>(v);
  if constexpr (sizeof(T) == 4) {
    const int x = l % Lx, y = (l / Lx) % Ly, z = l / (Lx * Ly);
    const float a = __ldg(s2p + x) + __ldg(s2p + kMaxL + y) + __ldg(s2p + 2 * kMaxL + z);
#pragma unroll
    for (int p = 0; p < L; ++p) {
      float k = c_over_V * __frcp_rn(a + s2t[p]);
      if (p == 0 && l == 0) k = 0.0f;
      v[p] = scale(v[p], (T)k);
    }
  } else {
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = scale(v[p], __ldg(kfac + (l + p * S)));
  }
  regfft::inverse<T, L>(v);
#pragma unroll
  for (int p = 0; p < L; ++p) line[p * S] = v[p];
}

template <class T, int L>
size_t xpass_smem() {
  return (size_t)xpass_lines<T, L>() * (L + 1) * sizeof(cx<T>);
}

#define LGF_AXIS_LENGTHS(X) X(4) X(6) X(8) X(12) X(16) X(20) X(24) X(32) X(48) X(64)

template <class T>
constexpr bool reg_ok(int L) {
  // FP64 lines longer than 32 would not fit in registers
  return sizeof(T) == 4 ? true : L <= 32;
}

template <class T, int L>
cudaError_t xpass_launch(void* D, int64_t V, int inverse, const DevState* st, cudaStream_t s) {
  const int64_t total = 4 * (V / L);
  constexpr int NL = xpass_lines<T, L>();
  const unsigned nb = (unsigned)((total + NL - 1) / NL);
  const size_t sm = xpass_smem<T, L>();
  if (inverse)
    launch_pdl(k_xpass<T, L, true>, nb, 128, sm, s, static_cast<cx<T>*>(D), total, st);
  else
    launch_pdl(k_xpass<T, L, false>, nb, 128, sm, s, static_cast<cx<T>*>(D), total, st);
  return cudaPeekAtLastError();
}

template <class T, int L>
cudaError_t strided_launch(void* D, int64_t V, int64_t S, int inverse, const DevState* st, cudaStream_t s) {
  const unsigned nb = (unsigned)((4 * (V / L) + 127) / 128);
  if (inverse)
    launch_pdl(k_strided<T, L, true>, nb, 128, 0, s, static_cast<cx<T>*>(D), V, S, st);
  else
    launch_pdl(k_strided<T, L, false>, nb, 128, 0, s, static_cast<cx<T>*>(D), V, S, st);
  return cudaPeekAtLastError();
}

template <class T, int L>
cudaError_t tpass_launch(void* D, int64_t V, int Lx, int Ly, const void* kfac, const float* s2p, float c_over_V,
                         const DevState* st, cudaStream_t s) {
  const unsigned nb = (unsigned)((4 * (V / L) + 127) / 128);
  launch_pdl(k_tpass<T, L>, nb, 128, 0, s, static_cast<cx<T>*>(D), V, Lx, Ly, static_cast<const T*>(kfac), s2p,
             c_over_V, st);
  return cudaPeekAtLastError();
}

template <class T>
cudaError_t set_xpass_smem_T() {
  cudaError_t e = cudaSuccess;
#define LGF_SET(L)                                                                                       \
  if (reg_ok<T>(L) && e == cudaSuccess) {                                                                \
    e = cudaFuncSetAttribute(k_xpass<T, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                             (int)xpass_smem<T, L>());                                                   \
    if (e == cudaSuccess)                                                                                \
      e = cudaFuncSetAttribute(k_xpass<T, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                               (int)xpass_smem<T, L>());                                                 \
  }
  if constexpr (sizeof(T) == 4) {
    LGF_AXIS_LENGTHS(LGF_SET)
  } else {
    LGF_SET(4) LGF_SET(6) LGF_SET(8) LGF_SET(12) LGF_SET(16) LGF_SET(20) LGF_SET(24) LGF_SET(32)
  }
#undef LGF_SET
  return e;
}

}  // namespace

bool axis_pass_supported(int prec, int L) {
  switch (L) {
    case 4: case 6: case 8: case 12: case 16: case 20: case 24: case 32:
      return true;
    case 48: case 64:
      return prec == 4;
    default:
      return false;
  }
}

cudaError_t axis_pass_init() {
  cudaError_t e = set_xpass_smem_T<float>();
  if (e == cudaSuccess) e = set_xpass_smem_T<double>();
  return e;
}

cudaError_t launch_xpass(int prec, int L, void* D, int64_t V, int inverse, const DevState* st, cudaStream_t s) {
#define LGF_CASE(N)                                                                \
  case N:                                                                          \
    if (prec == 4) return xpass_launch<float, N>(D, V, inverse, st, s);            \
    if constexpr (N <= 32) return xpass_launch<double, N>(D, V, inverse, st, s);   \
    break;
  switch (L) { LGF_AXIS_LENGTHS(LGF_CASE) }
#undef LGF_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_strided(int prec, int L, void* D, int64_t V, int64_t S, int inverse, const DevState* st,
                           cudaStream_t s) {
#define LGF_CASE(N)                                                                  \
  case N:                                                                            \
    if (prec == 4) return strided_launch<float, N>(D, V, S, inverse, st, s);         \
    if constexpr (N <= 32) return strided_launch<double, N>(D, V, S, inverse, st, s); \
    break;
  switch (L) { LGF_AXIS_LENGTHS(LGF_CASE) }
#undef LGF_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_tpass(int prec, int L, void* D, int64_t V, int Lx, int Ly, const void* kfac, const float* s2p,
                         float c_over_V, const DevState* st, cudaStream_t s) {
#define LGF_CASE(N)                                                                             \
  case N:                                                                                       \
    if (prec == 4) return tpass_launch<float, N>(D, V, Lx, Ly, kfac, s2p, c_over_V, st, s);     \
    if constexpr (N <= 32) return tpass_launch<double, N>(D, V, Lx, Ly, kfac, s2p, c_over_V, st, s); \
    break;
  switch (L) { LGF_AXIS_LENGTHS(LGF_CASE) }
#undef LGF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace lgf
