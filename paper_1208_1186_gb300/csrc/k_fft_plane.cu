// Fourier acceleration in three streaming passes, with the paper's "2D plus
// 2D" split of the 4D transform (Sec. 2.2) and in-register line FFTs
// (fft_reg.cuh):
//
//   k_plane_xy(fwd) -> k_plane_zt(fwd z, fwd t, x p2_max/(V p2), inv t, inv z)
//   -> k_plane_xy(inv)
//
// k_plane_xy: one CTA per (z, t) plane; the four fields of the plane
// (4 LX LY complex) are staged in shared memory by asynchronous copies (no
// register staging, all loads in flight at once); one thread per x-line does
// the x transforms, then one thread per y-line the y transforms.
// k_plane_zt (k_fft_zt.cu): the (z, t) transforms with the acceleration
// factor in between.
//
// Frequencies are left in digit-reversed order by the forward transforms and
// taken in that order by the inverse ones, so the acceleration factor is
// applied at digit-reversed positions (the same tables as the per-axis
// pipeline).  The packed gradient crosses memory three times per iteration
// instead of seven.
#include "fft_reg.cuh"
#include "lgf_df.cuh"
#include "lgf_gstep.cuh"
#include "lgf_kernels.cuh"

namespace lgf {

namespace {

// x-y planes with L <= 32 take the warp-tile kernel
constexpr bool kXyWarpTiles = true;
// FP32 gauge representation: the inverse x-y pass is fused with the G update,
// which loads G for kXyGstepSites sites at a time
constexpr bool kFuseXyinvGstep = true;
constexpr int kXyGstepSites = 4;

template <int LX, int LY>
constexpr int xy_threads() {
  return 4 * (LX > LY ? LX : LY);
}

// resident CTAs per SM asked of the register allocator: 4 x 128 threads at
// up to 128 registers for lines up to 32 complex in FP32
template <class T, int LX>
constexpr int xy_min_blocks() {
  return (sizeof(T) == 4 && LX <= 32) ? 4 : 1;
}

template <class T, int LX, int LY>
constexpr size_t xy_smem_bytes() {
  return (size_t)4 * LY * (LX + 1) * sizeof(cx<T>);
}

template <class T, int LX, int LY, bool INV>
__global__ void __launch_bounds__(xy_threads<LX, LY>(), xy_min_blocks<T, LX>()) k_plane_xy(cx<T>* __restrict__ D, int V,
                                                                   const DevState* __restrict__ st) {
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int NT = xy_threads<LX, LY>();
  constexpr int P = LX + 1;
  constexpr int N = LX * LY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw);  // [f][y][x], row pitch P
  const int plane = blockIdx.x * N;
  // stage the 4 planes (each contiguous in its field)
  static_assert((4 * N) % NT == 0, "tile must split evenly over the threads");
  constexpr int PER = 4 * N / NT;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = threadIdx.x + NT * k;
    const int f = i / N, q = i % N;
    cp_async_elem(tile + ((f * LY + q / LX) * P + q % LX), D + (f * V + plane + q));
  }
  cp_async_wait_all();
  __syncthreads();
  if (threadIdx.x < 4 * LY) {  // x lines
    cx<T>* row = tile + threadIdx.x * P;
    cx<T> v[LX];
#pragma unroll
    for (int p = 0; p < LX; ++p) v[p] = row[p];
    if (INV)
      regfft::inverse<T, LX>(v);
    else
      regfft::forward<T, LX>(v);
#pragma unroll
    for (int p = 0; p < LX; ++p) row[p] = v[p];
  }
  __syncthreads();
  if (threadIdx.x < 4 * LX) {  // y lines
    const int f = threadIdx.x / LX, x = threadIdx.x % LX;
    cx<T>* col = tile + f * LY * P + x;
    cx<T> v[LY];
#pragma unroll
    for (int p = 0; p < LY; ++p) v[p] = col[p * P];
    if (INV)
      regfft::inverse<T, LY>(v);
    else
      regfft::forward<T, LY>(v);
#pragma unroll
    for (int p = 0; p < LY; ++p) col[p * P] = v[p];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = threadIdx.x + NT * k;
    const int f = i / N, q = i % N;
    D[f * V + plane + q] = tile[(f * LY + q / LX) * P + q % LX];
  }
}

// x-y planes with L <= 32: a group of L lanes owns one (plane, field)
// tile from its load to its store, so a warp needs no CTA barrier and warps
// overlap their loads with one another's transforms.  Lane r loads y-line r
// straight into registers (for each y the group reads one contiguous row),
// transforms it, and one pass through shared memory hands it x-line r; a
// second pass turns the rows back into coalesced stores.  (The two 1D
// transforms commute, so y before x gives the same 2D transform.)  Four
// shared-memory accesses per element; one warp per CTA, floor(32 / L) tiles
// per warp (L <= 32; lanes past the last whole group idle through the
// transforms).
template <class T, int L>
constexpr int xyw_smem_bytes() {
  return (32 / L) * L * (L + 1) * (int)sizeof(cx<T>);
}

template <class T, int L, bool INV>
__global__ void __launch_bounds__(32) k_plane_xy_warp(cx<T>* __restrict__ D, int V, int ntiles,
                                                      const DevState* __restrict__ st) {
  static_assert(L <= 32, "a warp holds at least one tile");
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int G = 32 / L, P = L + 1, N = L * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / L, r = threadIdx.x % L;
  const int tile_id = blockIdx.x * G + g;  // = 4 plane + field
  // a group past the last tile, or past the last whole group of the warp,
  // idles but still takes part in every __syncwarp
  const bool active = g < G && tile_id < ntiles;
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw) + (active ? g : 0) * L * P;
  cx<T>* src = D + (active ? (tile_id & 3) * V + (tile_id >> 2) * N : 0);
  if (active) {  // y-line r from global, transformed, into column r
    cx<T> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = src[p * L + r];
    if (INV)
      regfft::inverse<T, L>(v);
    else
      regfft::forward<T, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[p * P + r] = v[p];
  }
  __syncwarp();
  if (active) {  // x-line r from row r
    cx<T> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = tile[r * P + p];
    if (INV)
      regfft::inverse<T, L>(v);
    else
      regfft::forward<T, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[r * P + p] = v[p];
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int k = 0; k < L; ++k) src[k * L + r] = tile[k * P + r];
  }
}

// x-y planes with 32 < L <= 64: the same scheme with one tile per CTA of two
// warps (thread r owns y-line r, then x-line r; CTA barriers between the
// phases).
template <class T, int L, bool INV>
__global__ void __launch_bounds__(64) k_plane_xy_pair(cx<T>* __restrict__ D, int V, int ntiles,
                                                      const DevState* __restrict__ st) {
  static_assert(L > 32 && L <= 64, "two warps per tile");
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int P = L + 1, N = L * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw);
  const int r = threadIdx.x, tile_id = blockIdx.x;  // = 4 plane + field
  const bool active = r < L;
  cx<T>* src = D + ((tile_id & 3) * V + (tile_id >> 2) * N);
  if (active) {
    cx<T> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = src[p * L + r];
    if (INV)
      regfft::inverse<T, L>(v);
    else
      regfft::forward<T, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[p * P + r] = v[p];
  }
  __syncthreads();
  if (active) {
    cx<T> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = tile[r * P + p];
    if (INV)
      regfft::inverse<T, L>(v);
    else
      regfft::forward<T, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[r * P + p] = v[p];
  }
  __syncthreads();
  for (int k = 0; k < L; ++k)
    if (active) src[k * L + r] = tile[k * P + r];
  (void)ntiles;
}

// Inverse x-y transform fused with the gauge step on G (FP32 gauge
// representation).  One CTA of four warps per floor(32 / L) planes (L <= 32): warp f inverse-
// transforms field f of the CTA's planes exactly as k_plane_xy_warp does and
// leaves Delta~ in shared memory (it is never written back: nothing reads it
// after the update); after one CTA barrier the 128 threads apply the gauge
// step to the planes' sites, Delta~ from shared memory, G streamed through
// registers.  The G stream of some CTAs overlaps the transforms of others.
template <int L, int NC, class RT, int KS>
__global__ void __launch_bounds__(128) k_plane_xyinv_gstep(const cx<float>* __restrict__ D, cx<float>* G, int V,
                                                           int nplanes, double hd, const DevState* __restrict__ st) {
  static_assert(L <= 32, "a warp holds at least one tile");
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int GP = 32 / L, P = L + 1, N = L * L, TS = L * P;  // planes per CTA, pitch, plane, tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tiles = reinterpret_cast<cx<float>*>(smem_raw);  // [field][plane of the CTA][y][x]
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / L, r = lane % L;
  const int plane0 = blockIdx.x * GP;
  const bool active = g < GP && plane0 + g < nplanes;
  cx<float>* tile = tiles + (f * GP + (active ? g : 0)) * TS;
  if (active) {  // inverse y-line r from global memory into column r
    const cx<float>* src = D + ((int64_t)f * V + (int64_t)(plane0 + g) * N);
    cx<float> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = src[p * L + r];
    regfft::inverse<float, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[p * P + r] = v[p];
  }
  __syncwarp();
  if (active) {  // inverse x-line r in row r
    cx<float> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = tile[r * P + p];
    regfft::inverse<float, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[r * P + p] = v[p];
  }
  __syncthreads();
  // KS sites per round: all their G loads are issued before any is used
  // (G is read and written through the same pointer, so the compiler would
  // not hoist a later site's loads above an earlier site's stores)
  const RT h = (RT)hd;
  const int np = nplanes - plane0 < GP ? nplanes - plane0 : GP;
  const int ns = np * N;
  const int64_t base = (int64_t)plane0 * N;
  for (int q0 = threadIdx.x; q0 < ns; q0 += KS * blockDim.x) {
    M3<float> Gk[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int q = q0 + k * blockDim.x;
      if (q < ns) Gk[k] = gstep_load_G<float, NC>(G, V, base + q);
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int q = q0 + k * blockDim.x;
      if (q < ns) {
        const int gi = q / N, qq = q - gi * N;
        const int o = gi * TS + (qq / L) * P + qq % L;
        gstep_store<float, NC, RT>(
            gstep_g<RT>(tiles[o], tiles[GP * TS + o], tiles[2 * GP * TS + o], tiles[3 * GP * TS + o], h), Gk[k], G,
            V, base + q);
      }
    }
  }
}

// The double-float tail's inverse x-y pass fused with its gauge step
// (tail_eta_site), as k_plane_xyinv_gstep fuses the FP32 phase's G update:
// four warps inverse-transform the four fields of the CTA's planes, Delta~
// stays in shared memory, and after one CTA barrier the 128 threads update
// 1 + eta at the planes' sites.  The transforms are those of
// k_plane_xy_warp, so the result is bit-identical to the unfused pass plus
// k_tail_eta_step.
template <int L>
__global__ void __launch_bounds__(128) k_plane_xyinv_eta(const cx<float>* __restrict__ D, cx<float>* __restrict__ eh,
                                                         cx<float>* __restrict__ el, int V, int nplanes, float h,
                                                         const DevState* __restrict__ st) {
  static_assert(L <= 32, "a warp holds at least one tile");
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int GP = 32 / L, P = L + 1, N = L * L, TS = L * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tiles = reinterpret_cast<cx<float>*>(smem_raw);  // [field][plane of the CTA][y][x]
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / L, r = lane % L;
  const int plane0 = blockIdx.x * GP;
  const bool active = g < GP && plane0 + g < nplanes;
  cx<float>* tile = tiles + (f * GP + (active ? g : 0)) * TS;
  if (active) {  // inverse y-line r from global memory into column r
    const cx<float>* src = D + ((int64_t)f * V + (int64_t)(plane0 + g) * N);
    cx<float> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = src[p * L + r];
    regfft::inverse<float, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[p * P + r] = v[p];
  }
  __syncwarp();
  if (active) {  // inverse x-line r in row r
    cx<float> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = tile[r * P + p];
    regfft::inverse<float, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[r * P + p] = v[p];
  }
  __syncthreads();
  const int np = nplanes - plane0 < GP ? nplanes - plane0 : GP;
  const int ns = np * N;
  const int base = plane0 * N;
  for (int q = threadIdx.x; q < ns; q += blockDim.x) {
    const int gi = q / N, qq = q - gi * N;
    const int o = gi * TS + (qq / L) * P + qq % L;
    tail_eta_site(tiles[o], tiles[GP * TS + o], tiles[2 * GP * TS + o], tiles[3 * GP * TS + o], h, eh, el, V,
                  base + q);
  }
}

template <int L>
constexpr size_t xyinv_gstep_smem() {
  return (size_t)4 * (L <= 32 ? 32 / L : 1) * L * (L + 1) * sizeof(cx<float>);
}

// The fused kernel for 32 < L <= 64: one plane per CTA of 256 threads, two
// warps per field for the transforms (CTA barriers between the phases), then
// all 256 threads on the gauge step.
template <int L, int NC, class RT, int KS>
__global__ void __launch_bounds__(256, 2) k_plane_xyinv_gstep_pair(const cx<float>* __restrict__ D, cx<float>* G,
                                                                int V, int nplanes, double hd,
                                                                const DevState* __restrict__ st) {
  static_assert(L > 32 && L <= 64, "two warps per field");
  pdl_wait();
  if (st != nullptr && st->done) return;
  constexpr int P = L + 1, N = L * L, TS = L * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tiles = reinterpret_cast<cx<float>*>(smem_raw);  // [field][y][x]
  const int f = threadIdx.x >> 6, r = threadIdx.x & 63;
  const int plane = blockIdx.x;
  const bool active = r < L;
  cx<float>* tile = tiles + f * TS;
  if (active) {
    const cx<float>* src = D + ((int64_t)f * V + (int64_t)plane * N);
    cx<float> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = src[p * L + r];
    regfft::inverse<float, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[p * P + r] = v[p];
  }
  __syncthreads();
  if (active) {
    cx<float> v[L];
#pragma unroll
    for (int p = 0; p < L; ++p) v[p] = tile[r * P + p];
    regfft::inverse<float, L>(v);
#pragma unroll
    for (int p = 0; p < L; ++p) tile[r * P + p] = v[p];
  }
  __syncthreads();
  const RT h = (RT)hd;
  const int64_t base = (int64_t)plane * N;
  for (int q0 = threadIdx.x; q0 < N; q0 += KS * blockDim.x) {
    M3<float> Gk[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int q = q0 + k * blockDim.x;
      if (q < N) Gk[k] = gstep_load_G<float, NC>(G, V, base + q);
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int q = q0 + k * blockDim.x;
      if (q < N) {
        const int o = (q / L) * P + q % L;
        gstep_store<float, NC, RT>(gstep_g<RT>(tiles[o], tiles[TS + o], tiles[2 * TS + o], tiles[3 * TS + o], h),
                                   Gk[k], G, V, base + q);
      }
    }
  }
  (void)nplanes;
}

template <int L>
constexpr size_t xyinv_gstep_pair_smem() {
  return (size_t)4 * L * (L + 1) * sizeof(cx<float>);
}

}  // namespace

namespace {

// instantiated x-y planes (LX = LY) and z-t planes (LZ, LT), per precision
#define LGF_XY_F32(X) X(4) X(6) X(8) X(12) X(16) X(20) X(24) X(32) X(48)
#define LGF_XY_F64(X) X(4) X(6) X(8) X(12) X(16) X(20) X(24) X(32)
template <class T, int L>
cudaError_t xy_launch(void* D, int64_t V, int inverse, const DevState* st, cudaStream_t s, int Lz, int Lt) {
  if constexpr (L <= 32 && kXyWarpTiles) {
    const int ntiles = 4 * Lz * Lt;
    const unsigned nb = (unsigned)((ntiles + 32 / L - 1) / (32 / L));
    constexpr int sm = xyw_smem_bytes<T, L>();
    const auto Dp = static_cast<cx<T>*>(D);
    if (inverse) return launch_pdl(k_plane_xy_warp<T, L, true>, nb, 32, sm, s, Dp, (int)V, ntiles, st);
    return launch_pdl(k_plane_xy_warp<T, L, false>, nb, 32, sm, s, Dp, (int)V, ntiles, st);
  } else if constexpr (L > 32 && L <= 64 && kXyWarpTiles) {
    const int ntiles = 4 * Lz * Lt;
    constexpr int sm = L * (L + 1) * (int)sizeof(cx<T>);
    const auto Dp = static_cast<cx<T>*>(D);
    if (inverse) return launch_pdl(k_plane_xy_pair<T, L, true>, (unsigned)ntiles, 64, sm, s, Dp, (int)V, ntiles, st);
    return launch_pdl(k_plane_xy_pair<T, L, false>, (unsigned)ntiles, 64, sm, s, Dp, (int)V, ntiles, st);
  }
  const unsigned nb = (unsigned)(Lz * Lt);
  constexpr int NT = xy_threads<L, L>();
  constexpr size_t sm = xy_smem_bytes<T, L, L>();
  const auto Dp = static_cast<cx<T>*>(D);
  if (inverse) return launch_pdl(k_plane_xy<T, L, L, true>, nb, NT, sm, s, Dp, (int)V, st);
  return launch_pdl(k_plane_xy<T, L, L, false>, nb, NT, sm, s, Dp, (int)V, st);
}

template <int L>
cudaError_t xyinv_gstep_pair_launch(int nc, bool r64, const cx<float>* D, cx<float>* G, int V, int nplanes,
                                    double ha, const DevState* st, cudaStream_t s) {
  const unsigned nb = (unsigned)nplanes;
  constexpr size_t sm = xyinv_gstep_pair_smem<L>();
  if (nc == 9) {
    if (r64) return launch_pdl(k_plane_xyinv_gstep_pair<L, 9, double, kXyGstepSites>, nb, 256, sm, s, D, G, V, nplanes, ha, st);
    return launch_pdl(k_plane_xyinv_gstep_pair<L, 9, float, kXyGstepSites>, nb, 256, sm, s, D, G, V, nplanes, ha, st);
  }
  if (r64) return launch_pdl(k_plane_xyinv_gstep_pair<L, 6, double, kXyGstepSites>, nb, 256, sm, s, D, G, V, nplanes, ha, st);
  return launch_pdl(k_plane_xyinv_gstep_pair<L, 6, float, kXyGstepSites>, nb, 256, sm, s, D, G, V, nplanes, ha, st);
}

template <int L>
cudaError_t xyinv_gstep_pair_attr() {
  constexpr int sm = (int)xyinv_gstep_pair_smem<L>();
  cudaError_t e = cudaFuncSetAttribute(k_plane_xyinv_gstep_pair<L, 9, double, kXyGstepSites>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_plane_xyinv_gstep_pair<L, 9, float, kXyGstepSites>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_plane_xyinv_gstep_pair<L, 6, double, kXyGstepSites>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_plane_xyinv_gstep_pair<L, 6, float, kXyGstepSites>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

template <int L>
cudaError_t xyinv_gstep_launch(int nc, bool r64, const cx<float>* D, cx<float>* G, int V, int nplanes, double ha,
                               const DevState* st, cudaStream_t s) {
  const unsigned nb = (unsigned)((nplanes + 32 / L - 1) / (32 / L));
  constexpr size_t sm = xyinv_gstep_smem<L>();
  if (nc == 9) {
    if (r64) return launch_pdl(k_plane_xyinv_gstep<L, 9, double, kXyGstepSites>, nb, 128, sm, s, D, G, V, nplanes, ha, st);
    return launch_pdl(k_plane_xyinv_gstep<L, 9, float, kXyGstepSites>, nb, 128, sm, s, D, G, V, nplanes, ha, st);
  }
  if (r64) return launch_pdl(k_plane_xyinv_gstep<L, 6, double, kXyGstepSites>, nb, 128, sm, s, D, G, V, nplanes, ha, st);
  return launch_pdl(k_plane_xyinv_gstep<L, 6, float, kXyGstepSites>, nb, 128, sm, s, D, G, V, nplanes, ha, st);
}

template <class T, int L>
cudaError_t xy_attr() {
  if constexpr (L <= 32) {
    cudaError_t e = cudaFuncSetAttribute(k_plane_xy_warp<T, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         xyw_smem_bytes<T, L>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_plane_xy_warp<T, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               xyw_smem_bytes<T, L>());
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaFuncSetAttribute(k_plane_xy<T, L, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)xy_smem_bytes<T, L, L>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_plane_xy<T, L, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)xy_smem_bytes<T, L, L>());
  return e;
}

}  // namespace

bool plane_pipeline_supported(int prec, int Lx, int Ly, int Lz, int Lt) {
  if (Lx != Ly) return false;
  if (Lx % (prec == 4 ? 4 : 2) != 0) return false;
  bool xy = false, zt = false;
#define LGF_XYQ(L) xy = xy || Lx == L;
#define LGF_ZTQ(A, B) zt = zt || (Lz == A && Lt == B);
  if (prec == 4) {
    LGF_XY_F32(LGF_XYQ)
    LGF_ZT_F32(LGF_ZTQ)
  } else {
    LGF_XY_F64(LGF_XYQ)
    LGF_ZT_F64(LGF_ZTQ)
  }
#undef LGF_XYQ
#undef LGF_ZTQ
  return xy && zt;
}

cudaError_t plane_pipeline_init() {
  cudaError_t e = cudaSuccess;
#define LGF_XYA32(L) \
  if (e == cudaSuccess) e = xy_attr<float, L>();
#define LGF_XYA64(L) \
  if (e == cudaSuccess) e = xy_attr<double, L>();
  if (e == cudaSuccess) e = xyinv_gstep_pair_attr<48>();
  LGF_XY_F32(LGF_XYA32)
  LGF_XY_F64(LGF_XYA64)
#undef LGF_XYA32
#undef LGF_XYA64
  if (e == cudaSuccess) e = plane_zt_init();
  if (e == cudaSuccess) e = plane_xyinv_eta_init();
  return e;
}

cudaError_t launch_plane_xy(int prec, int L, void* D, int64_t V, int Lz, int Lt, int inverse, const DevState* st,
                            cudaStream_t s) {
#define LGF_XY32(N) \
  if (L == N) return xy_launch<float, N>(D, V, inverse, st, s, Lz, Lt);
#define LGF_XY64(N) \
  if (L == N) return xy_launch<double, N>(D, V, inverse, st, s, Lz, Lt);
  if (prec == 4) {
    LGF_XY_F32(LGF_XY32)
  } else {
    LGF_XY_F64(LGF_XY64)
  }
#undef LGF_XY32
#undef LGF_XY64
  return cudaErrorInvalidValue;
}

bool plane_xyinv_eta_supported(int L) {
  switch (L) {
    case 4: case 6: case 8: case 12: case 16: case 20: case 24: case 32:
      return kFuseXyinvGstep;
    default:
      return false;
  }
}

cudaError_t plane_xyinv_eta_init() {
  cudaError_t e = cudaSuccess;
#define LGF_ETA_ATTR(L)                                                                           \
  if (e == cudaSuccess)                                                                           \
    e = cudaFuncSetAttribute(k_plane_xyinv_eta<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)xyinv_gstep_smem<L>());
  LGF_ETA_ATTR(4) LGF_ETA_ATTR(6) LGF_ETA_ATTR(8) LGF_ETA_ATTR(12) LGF_ETA_ATTR(16) LGF_ETA_ATTR(20) LGF_ETA_ATTR(24)
  LGF_ETA_ATTR(32)
#undef LGF_ETA_ATTR
  return e;
}

cudaError_t launch_plane_xyinv_eta(int L, const void* D, void* eta, int64_t V, int Lz, int Lt, double half_alpha,
                                   const DevState* st, cudaStream_t s) {
  const int nplanes = Lz * Lt;
  const auto Dp = static_cast<const cx<float>*>(D);
  auto e = static_cast<cx<float>*>(eta);
  const float h = (float)half_alpha;
#define LGF_ETA_L(N)                                                                                              \
  case N: {                                                                                                       \
    const unsigned nb = (unsigned)((nplanes + 32 / N - 1) / (32 / N));                                           \
    return launch_pdl(k_plane_xyinv_eta<N>, nb, 128, xyinv_gstep_smem<N>(), s, Dp, e, e + 9 * V, (int)V, nplanes, \
                      h, st);                                                                                     \
  }
  switch (L) {
    LGF_ETA_L(4) LGF_ETA_L(6) LGF_ETA_L(8) LGF_ETA_L(12) LGF_ETA_L(16) LGF_ETA_L(20) LGF_ETA_L(24) LGF_ETA_L(32)
    default:
      return cudaErrorInvalidValue;
  }
#undef LGF_ETA_L
}

bool plane_xyinv_gstep_supported(int prec, int L) {
  if (!kFuseXyinvGstep || prec != 4) return false;
  switch (L) {
    case 4: case 6: case 8: case 12: case 16: case 20: case 24: case 32: case 48:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_plane_xyinv_gstep(int L, int nc, const void* D, void* G, int64_t V, int Lz, int Lt,
                                     double half_alpha, bool reunit_fp64, const DevState* st, cudaStream_t s) {
  const int nplanes = Lz * Lt;
  const auto Dp = static_cast<const cx<float>*>(D);
  const auto Gp = static_cast<cx<float>*>(G);
  switch (L) {
    case 4: return xyinv_gstep_launch<4>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 6: return xyinv_gstep_launch<6>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 8: return xyinv_gstep_launch<8>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 12: return xyinv_gstep_launch<12>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 16: return xyinv_gstep_launch<16>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 20: return xyinv_gstep_launch<20>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 24: return xyinv_gstep_launch<24>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 32: return xyinv_gstep_launch<32>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    case 48: return xyinv_gstep_pair_launch<48>(nc, reunit_fp64, Dp, Gp, (int)V, nplanes, half_alpha, st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lgf
