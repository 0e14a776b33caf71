// z-t plane pass of the three-pass plane pipeline (k_fft_plane.cu holds the
// x-y passes): for every (field, y, run of BX consecutive x) one CTA holds
// the whole (z, t) plane of that run in shared memory and does
//   forward z, forward t, x p2_max / (V p2(k)) (0 at k = 0), inverse t,
//   inverse z
// (the middle of the paper's "2D plus 2D" transform, Sec. 2.2, with the
// Fourier acceleration of the steepest-descent step, Sec. 1, applied in
// between).  z lines are loaded from global memory into registers and
// transformed, handed to t lines through shared memory, and stored from
// registers after the inverse: four shared-memory accesses per element.
//
// Two schedule choices are template parameters, searched per lattice shape
// by the autotuner (lgf_autotune):
//   BX  the x-run width of a tile: 4 or 8 FP32 complex numbers (32 or 64
//       bytes per z load of a warp), 2 or 4 in FP64;
//   RO  the radix order of the z and t transforms (fft_reg.cuh): 0 greedy
//       (32 = 4 4 2), 1 the same factors reversed (32 = 2 4 4), 2 the pair
//       split (FP32): two threads share each line, the first radix-2 stage
//       runs across the pair with shuffles and each thread transforms its
//       half; half the registers per thread, twice the threads per tile.
// Frequencies stay in the forward transform's digit-reversed order and the
// inverse takes them in that order, so the acceleration factor is applied at
// digit-reversed positions: s2p holds, per radix order, 4 sin^2 of the
// frequency at each position of each axis (x and y always from order 0, the
// x-y pass's order; for order 2, the z factor at each z slot of the tile).
#include "fft_reg.cuh"
#include "lgf_kernels.cuh"

namespace lgf {

namespace {

// pitch of one t slice: BX*LZ plus padding that shifts consecutive t slices
// by one run of BX elements across the 32 shared-memory banks
template <class T, int LZ, int BX>
constexpr int zt_pitch() {
  constexpr int W = (int)sizeof(cx<T>) / 4;  // banks per element
  for (int pad = 0; pad < 32; ++pad)
    if ((((BX * LZ + pad) * W) % 32) == ((BX * W) % 32)) return BX * LZ + pad;
  return BX * LZ;
}

template <int LZ, int LT, int BX>
constexpr int zt_threads() {
  return BX * (LZ > LT ? LZ : LT);
}

// a thread holds a whole t line through the forward transform, the factor and
// the inverse: FP32 lines up to 32 run 3 CTAs of 128 threads per SM at BX = 4
// (up to 170 registers, no spills; 4 CTAs at 128 registers spilled 56 bytes
// per thread and took 22.6 instead of 21.7 us at 32^4, 5 and 6 CTAs took
// 23.9 and 28.9 us), 2 of 256 at BX = 8
template <class T, int LZ, int LT, int BX>
constexpr int zt_min_blocks() {
  return (sizeof(T) == 4 && LZ <= 32 && LT <= 32) ? (BX <= 4 ? 3 : 2) : 1;
}

template <class T, int LZ, int LT, int BX>
constexpr size_t zt_smem_bytes() {
  return (size_t)zt_pitch<T, LZ, BX>() * LT * sizeof(cx<T>);
}

// FP32: factor from s2p[RO][axis][position] and c_over_V = p2_max / V, 0 at
// k = 0.  FP64: per-site table kfac (an FP64 division per mode would be slow
// on this GPU; FP64 runs radix order 0 only).
template <class T, int LZ, int LT, int BX, int RO>
__global__ void __launch_bounds__(zt_threads<LZ, LT, BX>(), zt_min_blocks<T, LZ, LT, BX>())
    k_plane_zt(cx<T>* __restrict__ D, int Lx, int Ly, const T* __restrict__ kfac, const float* __restrict__ s2p,
               float c_over_V, const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int PT = zt_pitch<T, LZ, BX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw);  // [t][z][xb], t pitch PT
  const int nxr = Lx / BX;
  const int x0 = (blockIdx.x % nxr) * BX;
  const int y = blockIdx.x / nxr;
  const int f = blockIdx.y;
  const int LxLy = Lx * Ly;
  const int V = LxLy * LZ * LT;
  cx<T>* Df = D + (f * V + x0 + Lx * y);
  // forward z: line (xb, t) straight from global memory (for each z a warp
  // reads BX consecutive x at 32 / BX values of t: whole 32-byte sectors)
  if (threadIdx.x < BX * LT) {
    const int xb = threadIdx.x % BX, t = threadIdx.x / BX;
    cx<T>* line = tile + t * PT + xb;
    const cx<T>* g = Df + (xb + LxLy * LZ * t);
    cx<T> v[LZ];
#pragma unroll
    for (int p = 0; p < LZ; ++p) {  // running pointer: one address register
      v[p] = *g;
      g += LxLy;
    }
    regfft::forward<T, LZ, RO>(v);
#pragma unroll
    for (int p = 0; p < LZ; ++p) line[p * BX] = v[p];
  }
  __syncthreads();
  // t lines (xb, z): forward, acceleration factor, inverse
  if (threadIdx.x < BX * LZ) {
    const int xb = threadIdx.x % BX, z = threadIdx.x / BX;
    cx<T>* line = tile + z * BX + xb;
    cx<T> v[LT];
#pragma unroll
    for (int p = 0; p < LT; ++p) v[p] = line[p * PT];
    regfft::forward<T, LT, RO>(v);
    const int x = x0 + xb;
    if constexpr (sizeof(T) == 4) {
      // the t contribution at each position is a compile-time constant
      const float a = __ldg(s2p + x) + __ldg(s2p + kMaxL + y) + __ldg(s2p + RO * 4 * kMaxL + 2 * kMaxL + z);
      const bool origin = (x | y | z) == 0;
      regfft::static_for<0, LT>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        constexpr float s2t = (float)regfft::MomentumSq<LT, p, RO>::value;
        float kf = c_over_V * rcp_approx(a + s2t);
        if (p == 0 && origin) kf = 0.0f;
        v[p] = scale(v[p], (T)kf);
      });
    } else {
      static_assert(RO == 0, "FP64 z-t passes use radix order 0 (the per-site factor table's order)");
      const T* kl = kfac + (x + Lx * (y + Ly * z));
#pragma unroll
      for (int p = 0; p < LT; ++p) v[p] = scale(v[p], __ldg(kl + p * (LxLy * LZ)));
    }
    regfft::inverse<T, LT, RO>(v);
#pragma unroll
    for (int p = 0; p < LT; ++p) line[p * PT] = v[p];
  }
  __syncthreads();
  // inverse z, stored straight to global memory
  if (threadIdx.x < BX * LT) {
    const int xb = threadIdx.x % BX, t = threadIdx.x / BX;
    const cx<T>* line = tile + t * PT + xb;
    cx<T>* g = Df + (xb + LxLy * LZ * t);
    cx<T> v[LZ];
#pragma unroll
    for (int p = 0; p < LZ; ++p) v[p] = line[p * BX];
    regfft::inverse<T, LZ, RO>(v);
#pragma unroll
    for (int p = 0; p < LZ; ++p) {
      *g = v[p];
      g += LxLy;
    }
  }
}

// Radix order 2: the pair-split z and t transforms (FP32).  Thread 2 r + h
// holds half h of line r.  The forward z transform leaves element p of half h
// at z slot 2 p + h of the tile (frequency 2 digit_rev(Lz/2, p) + h), so that
// the two halves of a line sit in neighbouring slots; the t lines read and
// write their halves in natural order.
template <int LZ, int LT, int BX>
constexpr int zt_pair_threads() {
  return 2 * BX * (LZ > LT ? LZ : LT);
}

// 32 FP32 registers of line data per thread (L = 32): as many CTAs per SM as
// keep about 84 registers per thread (three 256-thread CTAs at L = 32, BX = 4:
// 24 warps)
template <int LZ, int LT, int BX>
constexpr int zt_pair_min_blocks() {
  constexpr int b = 65536 / (zt_pair_threads<LZ, LT, BX>() * 84);
  return b < 1 ? 1 : b;
}

template <int LZ, int LT, int BX>
__global__ void __launch_bounds__(zt_pair_threads<LZ, LT, BX>(), zt_pair_min_blocks<LZ, LT, BX>())
    k_plane_zt_pair(cx<float>* __restrict__ D, int Lx, int Ly, const float* __restrict__ s2p, float c_over_V,
                    const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int PT = zt_pitch<float, LZ, BX>();
  constexpr int HZ = LZ / 2, HT = LT / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tile = reinterpret_cast<cx<float>*>(smem_raw);  // [t][z slot][xb], t pitch PT
  const int nxr = Lx / BX;
  const int x0 = (blockIdx.x % nxr) * BX;
  const int y = blockIdx.x / nxr;
  const int f = blockIdx.y;
  const int LxLy = Lx * Ly;
  const int V = LxLy * LZ * LT;
  cx<float>* Df = D + (f * V + x0 + Lx * y);
  const int h = threadIdx.x & 1, r = threadIdx.x >> 1;
  // forward z: half h of line (xb, t) from global memory (the condition is
  // uniform over each warp: 2 BX LT is a multiple of 32)
  if (r < BX * LT) {
    const int xb = r % BX, t = r / BX;
    const cx<float>* g = Df + (xb + LxLy * (h * HZ) + LxLy * LZ * t);
    cx<float> v[HZ];
#pragma unroll
    for (int p = 0; p < HZ; ++p) {
      v[p] = *g;
      g += LxLy;
    }
    regfft::forward_pair<float, LZ>(v, h);
    cx<float>* line = tile + t * PT + h * BX + xb;
#pragma unroll
    for (int p = 0; p < HZ; ++p) line[2 * p * BX] = v[p];
  }
  __syncthreads();
  // t lines (xb, z slot): forward, acceleration factor, inverse
  if (r < BX * LZ) {
    const int xb = r % BX, zs = r / BX;
    cx<float>* line = tile + (h * HT) * PT + zs * BX + xb;
    cx<float> v[HT];
#pragma unroll
    for (int p = 0; p < HT; ++p) v[p] = line[p * PT];
    regfft::forward_pair<float, LT>(v, h);
    const int x = x0 + xb;
    const float a = __ldg(s2p + x) + __ldg(s2p + kMaxL + y) + __ldg(s2p + 2 * 4 * kMaxL + 2 * kMaxL + zs);
    const bool origin = (x | y | zs | h) == 0;  // z slot 0 and half 0 hold frequency 0
    regfft::static_for<0, HT>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      constexpr float s0 = (float)regfft::MomentumSqPair<LT, p, 0>::value;
      constexpr float s1 = (float)regfft::MomentumSqPair<LT, p, 1>::value;
      float kf = c_over_V * rcp_approx(a + (h ? s1 : s0));
      if (p == 0 && origin) kf = 0.0f;
      v[p] = scale(v[p], kf);
    });
    regfft::inverse_pair<float, LT>(v, h);
#pragma unroll
    for (int p = 0; p < HT; ++p) line[p * PT] = v[p];
  }
  __syncthreads();
  // inverse z, stored straight to global memory
  if (r < BX * LT) {
    const int xb = r % BX, t = r / BX;
    const cx<float>* line = tile + t * PT + h * BX + xb;
    cx<float> v[HZ];
#pragma unroll
    for (int p = 0; p < HZ; ++p) v[p] = line[2 * p * BX];
    regfft::inverse_pair<float, LZ>(v, h);
    cx<float>* g = Df + (xb + LxLy * (h * HZ) + LxLy * LZ * t);
#pragma unroll
    for (int p = 0; p < HZ; ++p) {
      *g = v[p];
      g += LxLy;
    }
  }
}

// the x-run widths instantiated per precision (the first is the default)
template <class T>
constexpr int zt_bx_default() {
  return sizeof(T) == 4 ? 4 : 2;
}
template <class T>
constexpr int zt_bx_wide() {
  return 2 * zt_bx_default<T>();
}

// radix order 1 is instantiated only where it changes the z or t stages
template <class T, int LZ, int LT>
constexpr bool zt_has_ro1() {
  return sizeof(T) == 4 && (regfft::orders_differ(LZ) || regfft::orders_differ(LT));
}

// radix order 2 (pair split) for FP32 lines with at least one extent >= 16
// (the shorter lines fit their registers anyway) and warp-aligned phases
template <class T, int LZ, int LT>
constexpr bool zt_has_ro2() {
  return sizeof(T) == 4 && (LZ >= 16 || LT >= 16) && regfft::pair_supported(LZ) && regfft::pair_supported(LT) &&
         (2 * 4 * LZ) % 32 == 0 && (2 * 4 * LT) % 32 == 0;
}

template <int LZ, int LT, int BX>
constexpr size_t zt_pair_smem_bytes() {
  return (size_t)zt_pitch<float, LZ, BX>() * LT * sizeof(cx<float>);
}

template <class T, int LZ, int LT, int BX, int RO>
cudaError_t zt_launch_one(void* D, int Lx, int Ly, const void* kfac, const float* s2p, float c_over_V,
                          const DevState* st, cudaStream_t s) {
  dim3 grid((unsigned)((Lx / BX) * Ly), 4);
  return launch_pdl(k_plane_zt<T, LZ, LT, BX, RO>, grid, zt_threads<LZ, LT, BX>(), zt_smem_bytes<T, LZ, LT, BX>(),
                    s, static_cast<cx<T>*>(D), Lx, Ly, static_cast<const T*>(kfac), s2p, c_over_V, st);
}

template <int LZ, int LT, int BX>
cudaError_t zt_launch_pair(void* D, int Lx, int Ly, const float* s2p, float c_over_V, const DevState* st,
                           cudaStream_t s) {
  dim3 grid((unsigned)((Lx / BX) * Ly), 4);
  return launch_pdl(k_plane_zt_pair<LZ, LT, BX>, grid, zt_pair_threads<LZ, LT, BX>(),
                    zt_pair_smem_bytes<LZ, LT, BX>(), s, static_cast<cx<float>*>(D), Lx, Ly, s2p, c_over_V, st);
}

template <class T, int LZ, int LT>
cudaError_t zt_launch(void* D, int Lx, int Ly, const void* kfac, const float* s2p, float c_over_V, int bx, int ro,
                      const DevState* st, cudaStream_t s) {
  constexpr int B0 = zt_bx_default<T>(), B1 = zt_bx_wide<T>();
  if (bx == 0) bx = B0;
  if (bx != B0 && bx != B1) return cudaErrorInvalidValue;
  if (Lx % bx != 0) return cudaErrorInvalidValue;
  if (ro == 2) {
    if constexpr (zt_has_ro2<T, LZ, LT>()) {
      if (bx == B0) return zt_launch_pair<LZ, LT, B0>(D, Lx, Ly, s2p, c_over_V, st, s);
      return zt_launch_pair<LZ, LT, B1>(D, Lx, Ly, s2p, c_over_V, st, s);
    }
    return cudaErrorInvalidValue;
  }
  if (ro == 1) {
    if constexpr (zt_has_ro1<T, LZ, LT>()) {
      if (bx == B0) return zt_launch_one<T, LZ, LT, B0, 1>(D, Lx, Ly, kfac, s2p, c_over_V, st, s);
      return zt_launch_one<T, LZ, LT, B1, 1>(D, Lx, Ly, kfac, s2p, c_over_V, st, s);
    }
    return cudaErrorInvalidValue;
  }
  if (ro != 0) return cudaErrorInvalidValue;
  if (bx == B0) return zt_launch_one<T, LZ, LT, B0, 0>(D, Lx, Ly, kfac, s2p, c_over_V, st, s);
  return zt_launch_one<T, LZ, LT, B1, 0>(D, Lx, Ly, kfac, s2p, c_over_V, st, s);
}

template <class T, int LZ, int LT, int BX, int RO>
cudaError_t zt_attr_one() {
  return cudaFuncSetAttribute(k_plane_zt<T, LZ, LT, BX, RO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)zt_smem_bytes<T, LZ, LT, BX>());
}

template <class T, int LZ, int LT>
cudaError_t zt_attr() {
  constexpr int B0 = zt_bx_default<T>(), B1 = zt_bx_wide<T>();
  cudaError_t e = zt_attr_one<T, LZ, LT, B0, 0>();
  if (e == cudaSuccess) e = zt_attr_one<T, LZ, LT, B1, 0>();
  if constexpr (zt_has_ro1<T, LZ, LT>()) {
    if (e == cudaSuccess) e = zt_attr_one<T, LZ, LT, B0, 1>();
    if (e == cudaSuccess) e = zt_attr_one<T, LZ, LT, B1, 1>();
  }
  if constexpr (zt_has_ro2<T, LZ, LT>()) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_plane_zt_pair<LZ, LT, B0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)zt_pair_smem_bytes<LZ, LT, B0>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_plane_zt_pair<LZ, LT, B1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)zt_pair_smem_bytes<LZ, LT, B1>());
  }
  return e;
}

}  // namespace

cudaError_t plane_zt_init() {
  cudaError_t e = cudaSuccess;
#define LGF_ZTA32(A, B) \
  if (e == cudaSuccess) e = zt_attr<float, A, B>();
#define LGF_ZTA64(A, B) \
  if (e == cudaSuccess) e = zt_attr<double, A, B>();
  LGF_ZT_F32(LGF_ZTA32)
  LGF_ZT_F64(LGF_ZTA64)
#undef LGF_ZTA32
#undef LGF_ZTA64
  return e;
}

bool plane_zt_schedule_supported(int prec, int Lx, int Lz, int Lt, int bx, int ro) {
  const int b0 = prec == 4 ? 4 : 2;
  if (bx != 0 && bx != b0 && bx != 2 * b0) return false;
  if (Lx % (bx == 0 ? b0 : bx) != 0) return false;
  if (ro == 0) return true;
  if (prec != 4) return false;
  if (ro == 1) return regfft::orders_differ(Lz) || regfft::orders_differ(Lt);
  if (ro != 2) return false;
  bool inst = false;
#define LGF_ZTR2(A, B) \
  if (Lz == A && Lt == B) inst = zt_has_ro2<float, A, B>();
  LGF_ZT_F32(LGF_ZTR2)
#undef LGF_ZTR2
  return inst;
}

cudaError_t launch_plane_zt(int prec, int Lx, int Ly, int Lz, int Lt, void* D, const void* kfac, const float* s2p,
                            float c_over_V, int bx, int ro, const DevState* st, cudaStream_t s) {
#define LGF_ZT32(A, B) \
  if (Lz == A && Lt == B) return zt_launch<float, A, B>(D, Lx, Ly, kfac, s2p, c_over_V, bx, ro, st, s);
#define LGF_ZT64(A, B) \
  if (Lz == A && Lt == B) return zt_launch<double, A, B>(D, Lx, Ly, kfac, s2p, c_over_V, bx, ro, st, s);
  if (prec == 4) {
    LGF_ZT_F32(LGF_ZT32)
  } else {
    LGF_ZT_F64(LGF_ZT64)
  }
#undef LGF_ZT32
#undef LGF_ZT64
  return cudaErrorInvalidValue;
}

}  // namespace lgf
