// Learned warm start: a 4D convolutional network that predicts, from the
// loaded links, an initial gauge transformation g0 = exp(sum_a c_a i
// lambda_a / 2) per site; the plain method then starts from G = g0 (gauge
// representation) and remains the judge through theta and F.
//
// Network: three 3^4-tap periodic convolutions, 48 -> 32 -> 32 -> 8 channels,
// ReLU after the first two; BF16 weights and activations, FP32 accumulation
// on the tensor cores (the forward and backward-data convolutions as
// tcgen05 implicit GEMMs, the weight gradient on warp-level 16x16x16 BF16
// tiles), FP32 master weights and Adam moments.  Training signal: the loss is -F(U^{g0}) (the
// method's own functional), whose derivative along left translations of
// g0(x) is the projection of the transformed links' gradient Delta'(x) onto
// the su(3) generators; Delta' comes from the gauge-representation gradient
// kernel with G = g0.
//
// Layouts: activations [site][channel] (BF16, channels fastest), weights
// [tap][in][out] with tap = ((dt*3 + dz)*3 + dy)*3 + dx, offsets d - 1.
#include <cuda_bf16.h>
#include <mma.h>

#include "lgf_kernels.cuh"

namespace lgf {
namespace warm {

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

constexpr int kFeat = 48;  // 32 link coefficients + 6 plaquettes + 10 zeros
constexpr int kHid = 32;
constexpr int kOut = 8;
constexpr int kOutPad = 16;  // the last layer is computed 16 wide, 8 used

namespace {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// su(3) coefficients of the traceless anti-Hermitian part of U, in the
// Gell-Mann basis with generators i lambda_a / 2 (c_a = -i Tr lambda_a A):
// written out entry by entry.
__device__ __forceinline__ void su3_coeffs(const M3<float>& u, float* c) {
  c[0] = u.e[0][1].im + u.e[1][0].im;
  c[1] = u.e[0][1].re - u.e[1][0].re;
  c[2] = u.e[0][0].im - u.e[1][1].im;
  c[3] = u.e[0][2].im + u.e[2][0].im;
  c[4] = u.e[0][2].re - u.e[2][0].re;
  c[5] = u.e[1][2].im + u.e[2][1].im;
  c[6] = u.e[1][2].re - u.e[2][1].re;
  c[7] = (u.e[0][0].im + u.e[1][1].im - 2.0f * u.e[2][2].im) * 0.57735026918962576451f;  // 1/sqrt(3)
}

template <int NC>
__global__ void __launch_bounds__(128) k_features(const cx<float>* __restrict__ U, bf16* __restrict__ x,
                                                  const Geom geo) {
  const int V = (int)geo.V;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords_i(geo.L, s, c);
  float f[kFeat];
#pragma unroll
  for (int i = 0; i < kFeat; ++i) f[i] = 0.0f;
  M3<float> u[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    u[mu] = load_m3i<float, NC>(U + mu * NC * V, V, s);
    su3_coeffs(u[mu], f + 8 * mu);
  }
  int k = 32;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int nu = mu + 1; nu < 4; ++nu) {
      const int sm = c[mu] < geo.L[mu] - 1 ? s + (int)geo.stride[mu] : s - (geo.L[mu] - 1) * (int)geo.stride[mu];
      const int sn = c[nu] < geo.L[nu] - 1 ? s + (int)geo.stride[nu] : s - (geo.L[nu] - 1) * (int)geo.stride[nu];
      const M3<float> un = load_m3i<float, NC>(U + nu * NC * V, V, sm);  // U_nu(x + mu)
      const M3<float> um = load_m3i<float, NC>(U + mu * NC * V, V, sn);  // U_mu(x + nu)
      M3<float> w1, w2;
      mm<float, 3>(w1, u[mu], un);
      mm<float, 3>(w2, u[nu], um);
      // Re Tr(w1 w2^dag) = sum Re(w1_ij conj(w2_ij))
      float tr = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) tr += w1.e[i][j].re * w2.e[i][j].re + w1.e[i][j].im * w2.e[i][j].im;
      f[k++] = tr * (1.0f / 3.0f);
    }
  bf16* out = x + (size_t)s * kFeat;
#pragma unroll
  for (int i = 0; i < kFeat; i += 2) {
    *reinterpret_cast<__nv_bfloat162*>(out + i) = __floats2bfloat162_rn(f[i], f[i + 1]);
  }
}

// ---------------------------------------------------------------------------
// g0 = exp(sum_a c_a i lambda_a / 2): Taylor series after scaling by 2^-s
// (norm below 1/2), s squarings, then reunitarisation.  Output: NC planes
// (the layout of the handle's accumulated transformation G).
// ---------------------------------------------------------------------------
__device__ __forceinline__ M3<float> algebra(const float* c) {
  const float r3 = 0.57735026918962576451f;
  M3<float> X;
  // X = (i/2) sum_a c_a lambda_a
  X.e[0][0] = mk<float>(0.f, 0.5f * (c[2] + r3 * c[7]));
  X.e[1][1] = mk<float>(0.f, 0.5f * (-c[2] + r3 * c[7]));
  X.e[2][2] = mk<float>(0.f, 0.5f * (-2.f * r3 * c[7]));
  X.e[0][1] = mk<float>(0.5f * c[1], 0.5f * c[0]);   // (i/2)(c1 - i c2)
  X.e[1][0] = mk<float>(-0.5f * c[1], 0.5f * c[0]);  // (i/2)(c1 + i c2)
  X.e[0][2] = mk<float>(0.5f * c[4], 0.5f * c[3]);
  X.e[2][0] = mk<float>(-0.5f * c[4], 0.5f * c[3]);
  X.e[1][2] = mk<float>(0.5f * c[6], 0.5f * c[5]);
  X.e[2][1] = mk<float>(-0.5f * c[6], 0.5f * c[5]);
  return X;
}

template <int NC>
__global__ void __launch_bounds__(128) k_expmap(const float* __restrict__ cin, int ldc, cx<float>* __restrict__ G,
                                                int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  float c[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) c[a] = cin[(size_t)s * ldc + a];
  M3<float> X = algebra(c);
  float n2 = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) n2 += norm2(X.e[i][j]);
  int sq = 0;
  float scl = 1.0f;
  while (n2 * scl * scl > 0.25f && sq < 30) {
    scl *= 0.5f;
    ++sq;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) X.e[i][j] = scale(X.e[i][j], scl);
  // Horner: E = I + X/1 (I + X/2 (... (I + X/10)))
  M3<float> E;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) E.e[i][j] = mk<float>(i == j ? 1.f : 0.f, 0.f);
#pragma unroll 1
  for (int k = 10; k >= 1; --k) {
    M3<float> T;
    mm<float, 3>(T, X, E);
    const float inv = 1.0f / (float)k;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) E.e[i][j] = mk<float>((i == j ? 1.f : 0.f) + inv * T.e[i][j].re, inv * T.e[i][j].im);
  }
  for (int q = 0; q < sq; ++q) {
    M3<float> T;
    mm<float, 3>(T, E, E);
    E = T;
  }
  reunitarize(E);
#pragma unroll
  for (int q = 0; q < NC; ++q) G[q * V + s] = E.e[q / 3][q % 3];
}

// ---------------------------------------------------------------------------
// training signal: dL/dc_a = -<i lambda_a / 2, Delta'> / (24 V) from the
// packed gradient D of the transformed links; written as BF16 [V][16]
// (channels 8..15 zero) scaled by `gain` (a power of two keeping the BF16
// values in range; the optimiser is scale invariant).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_signal(const cx<float>* __restrict__ D, int V, float coef,
                                                bf16* __restrict__ gc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const cx<float> d01 = D[s], d02 = D[V + s], d12 = D[2 * V + s], dd = D[3 * V + s];
  float p[16];
  p[0] = d01.im;
  p[1] = d01.re;
  p[2] = 0.5f * (dd.re - dd.im);
  p[3] = d02.im;
  p[4] = d02.re;
  p[5] = d12.im;
  p[6] = d12.re;
  p[7] = 0.86602540378443864676f * (dd.re + dd.im);  // sqrt(3)/2
#pragma unroll
  for (int a = 8; a < 16; ++a) p[a] = 0.f;
  bf16* out = gc + (size_t)s * kOutPad;
#pragma unroll
  for (int a = 0; a < 16; a += 2) *reinterpret_cast<__nv_bfloat162*>(out + a) = __floats2bfloat162_rn(coef * p[a], coef * p[a + 1]);
}

// ---------------------------------------------------------------------------
// convolutions on the tensor cores
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapc(int c, int d, int L) {
  int v = c + d;
  v = v < 0 ? v + L : v;
  return v >= L ? v - L : v;
}

// neighbour of site s (coordinates c) at tap offset (sign * (d - 1))
__device__ __forceinline__ int tap_site(const Geom& geo, const int c[4], int tap, int sign) {
  const int d0 = sign * (tap % 3 - 1), d1 = sign * ((tap / 3) % 3 - 1);
  const int d2 = sign * ((tap / 9) % 3 - 1), d3 = sign * (tap / 27 - 1);
  return wrapc(c[0], d0, geo.L[0]) +
         geo.L[0] * (wrapc(c[1], d1, geo.L[1]) + geo.L[1] * (wrapc(c[2], d2, geo.L[2]) + geo.L[2] * wrapc(c[3], d3, geo.L[3])));
}

// ---------------------------------------------------------------------------
// convolutions on the 5th-generation tensor cores (tcgen05): implicit GEMM
//   D[m, n] = sum_tap sum_k A_tap[m, k] B_tap[n, k],  A_tap[m, k] = act[site(m) + SIGN off(tap), k]
// with M = 128 output rows per CTA, N = the output channels and K = the
// gathered channels of one tap (16 per instruction).  Forward: act = x,
// B_tap = W^T (K-major copy [tap][out][in]), bias and ReLU in the epilogue.
// Backward data: act = gy, SIGN = -1, B_tap = W[tap][in][out] (already
// K-major in the output channels), the ReLU mask of the layer below in the
// epilogue.
//
// Rows.  The M rows of a CTA are 128 consecutive rows of the lattice laid
// out with a periodic halo in x and y: each (z, t) plane is (Ly + 2) lines of
// Lx + 2 rows (x = Lx-1, 0, ..., Lx-1, 0 along a line, the same wrap for the
// lines in y); rows on a halo are computed and discarded.  For an output row
// off the halo, the taps (dx, dy) read the rows dx + dy (Lx + 2) away, which
// stay inside its own plane.  So the nine taps of one (dz, dt) read a single
// window of gathered rows -- the CTA's 128 and Lx + 3 on each side -- at
// start addresses that differ by whole rows: for each of the 9 (dz, dt) the
// CTA gathers one window at plane offset SIGN (dz, dt) (each window row
// mapped on its own, so windows may cross planes), and its 9 taps' MMAs start
// (Lx + 3 + SIGN (dx + dy (Lx + 2))) rows into it.
//
// Shared memory, per pipeline stage: the window and the nine taps' B tiles,
// each "chunk-major" K-major -- 16-byte chunk c of row r at c * ROWS * 16 +
// r * 16 -- which is the no-swizzle canonical layout with SBO = 128 (the next
// 8 rows) and LBO = ROWS * 16 (the next 8 channels).  A warp's 32 rows of one
// chunk are 512 contiguous bytes, so the gathers write shared memory without
// bank conflicts.  ROWS, and with it the stage size, follows Lx.
//
// Pipeline: kTcStages stages; all 128 threads gather (cp.async, L1-cached:
// neighbouring windows overlap), one thread copies the group's B tiles (one
// bulk copy: the weights are stored in the tiles' order) and issues the
// 9 K/16 MMAs of a group into the FP32 accumulator in tensor memory (128
// lanes x N columns) and commits them to the stage's mbarrier.  A group's
// MMAs are issued before the previous group's stage is waited for and
// refilled, so the tensor core always has work queued.  Epilogue: each warp
// reads its 32 lanes with tcgen05.ld.  Every wait is bounded: on expiry the
// CTA records an error in err[0], stops issuing, waits (bounded) for its
// MMAs, frees its tensor memory and returns.  err[1] holds the poll budget of
// the stage waits (kConvWaitPolls unless lgf_net_set_wait_budget changed it).
// ---------------------------------------------------------------------------
constexpr int kTcStages = 2;
constexpr int kTcThreads = 160;  // four producer warps and the issuing warp
constexpr int kTcGroups = 9;  // (dz, dt) windows per CTA
constexpr int kTcTmemCols = 32;
constexpr unsigned kTcWaitLimit = (unsigned)kConvWaitPolls;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; lbo = bytes to the
// next 16-byte chunk along K, sbo = bytes to the next 8-row group
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;
}

// instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32
// accumulator, M = 128, N
template <int N>
constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// bounded wait (at most `polls` polls) for the phase of parity `parity` of an
// mbarrier; true if done
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned polls) {
  uint32_t done = 0;
  for (unsigned it = 0; it < polls && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// the same, giving up early once another thread of the CTA has set *stop
__device__ __forceinline__ bool mbar_wait_or_stop(uint64_t* bar, uint32_t parity, unsigned polls,
                                                  const volatile int* stop) {
  uint32_t done = 0;
  for (unsigned it = 0; it < polls && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (!done && *stop) break;
  }
  return done != 0;
}

// 16-byte asynchronous copy global -> shared, cached in L1 (.ca): the rows a
// CTA gathers for neighbouring groups overlap, and L1 serves the repeats
__device__ __forceinline__ void cp_async16(uint32_t sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sdst), "l"(gsrc) : "memory");
}

// window rows of a CTA: its 128 and Lx + 3 on each side, rounded up to whole
// 8-row groups
__host__ __device__ constexpr int tc_window_rows(int Lx) { return (128 + 2 * (Lx + 3) + 7) & ~7; }

template <int K, int N>
__host__ __device__ constexpr int tc_stage_bytes(int Lx) {
  return (tc_window_rows(Lx) + 9 * N) * K * 2;
}

__device__ __forceinline__ int wrap_add(int c, int d, int L) {
  int v = c + d;
  return v < 0 ? v + L : (v >= L ? v - L : v);
}

template <int K, int N, int SIGN, bool FWD>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(const bf16* __restrict__ act, const bf16* __restrict__ Wk,
                                                 const float* __restrict__ bias, const bf16* __restrict__ mask,
                                                 bf16* __restrict__ y, float* __restrict__ yf, const Geom geo,
                                                 bool relu, int* __restrict__ err) {
  static_assert(K % 16 == 0 && (N == 16 || N == 32), "tile shapes of this kernel");
  constexpr int NCH = K / 8;                         // 16-byte chunks per row
  constexpr int B_LBO = N * 16;                      // next chunk of a B tile
  constexpr int B_TAP = NCH * B_LBO;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kTcStages];   // a stage's window has landed (128 producer arrivals)
  __shared__ __align__(8) uint64_t empty[kTcStages];  // the MMAs reading a stage have completed
  __shared__ __align__(8) uint64_t bbars[kTcStages];  // a stage's B tiles have landed
  __shared__ __align__(8) uint64_t done_bar;          // all MMAs have completed
  __shared__ uint32_t tmem_slot;
  __shared__ int stop, last_issued;
  const int t = threadIdx.x, w = t >> 5;
  // roles: threads 0-127 gather the windows and write the output rows; lane 0
  // of warp 4 copies the B tiles and issues the MMAs
  const bool producer = t < 128;
  const bool issuer = t == 128;
  const int Lx = geo.L[0], Ly = geo.L[1], Lz = geo.L[2], Lt = geo.L[3];
  const int LXP = Lx + 2, LYP = Ly + 2;
  const int PLANE = LXP * LYP;             // padded rows of one (z, t) plane
  const int PR = PLANE * Lz * Lt;          // padded rows
  const int WR = 128 + 2 * (LXP + 1);      // window rows
  const uint32_t A_LBO = (uint32_t)tc_window_rows(Lx) * 16;  // next chunk of the window
  const uint32_t A_BYTES = NCH * A_LBO;
  const uint32_t STAGE = (uint32_t)tc_stage_bytes<K, N>(Lx);
  const int P0 = blockIdx.x * 128;
  // this thread's output row
  int s_out = -1;
  if (producer) {
    const int P = P0 + t;
    if (P < PR) {
      const int l = P / PLANE, r = P - l * PLANE;
      const int yp = r / LXP, xp = r - yp * LXP;
      if (xp >= 1 && xp <= Lx && yp >= 1 && yp <= Ly) s_out = (xp - 1) + Lx * ((yp - 1) + Ly * l);
    }
  }
  // this thread's window rows b = t + 128 k (b < WR; at most 3 for Lx <= 64):
  // padded row P0 - LXP - 1 + b as (x, y, z, t) of its source site, or absent
  constexpr int kRowsPerThread = 3;
  int rx[kRowsPerThread], ry[kRowsPerThread], rz[kRowsPerThread], rt[kRowsPerThread];
  bool rv[kRowsPerThread];
#pragma unroll
  for (int k = 0; k < kRowsPerThread; ++k) {
    const int b = t + 128 * k;
    const int P = P0 - LXP - 1 + b;
    rv[k] = producer && b < WR && P >= 0 && P < PR;
    rx[k] = ry[k] = rz[k] = rt[k] = 0;
    if (rv[k]) {
      const int l = P / PLANE, r = P - l * PLANE;
      const int yp = r / LXP, xp = r - yp * LXP;
      rx[k] = xp == 0 ? Lx - 1 : (xp == Lx + 1 ? 0 : xp - 1);
      ry[k] = yp == 0 ? Ly - 1 : (yp == Ly + 1 ? 0 : yp - 1);
      rz[k] = l % Lz;
      rt[k] = l / Lz;
    }
  }
  const uint32_t sbase = smem_u32(smem_raw);
  if (t == 0) {
    for (int k = 0; k < kTcStages; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&full[k])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[k])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bbars[k])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
    last_issued = -1;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // the stage waits' poll budget (err[1]); the final wait for the MMAs always
  // has the full budget, so that no MMA is in flight when the CTA frees its
  // tensor memory
  const unsigned stage_polls = (unsigned)err[1];

  // a thread whose wait expired records the error and stops the CTA: every
  // other wait of the CTA watches `stop` and gives up too
  auto fail = [&]() {
    atomicExch(err, 1);
    *(volatile int*)&stop = 1;
  };
  // gather group g = (dz, dt) into stage g % kTcStages: this thread's window
  // rows (zeros where a padded row lies outside the lattice)
  auto fill = [&](int g) {
    const uint32_t st = sbase + (g % kTcStages) * STAGE;
    const int dz = SIGN * (g % 3 - 1), dt = SIGN * (g / 3 - 1);
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
      const int b = t + 128 * k;
      if (b >= WR) break;
      const uint32_t dst = st + b * 16;
      if (rv[k]) {
        const int src = rx[k] + Lx * (ry[k] + Ly * (wrap_add(rz[k], dz, Lz) + Lz * wrap_add(rt[k], dt, Lt)));
        const bf16* p = act + (size_t)src * K;
#pragma unroll
        for (int c = 0; c < NCH; ++c) cp_async16(dst + c * A_LBO, p + c * 8);
      } else {
#pragma unroll
        for (int c = 0; c < NCH; ++c)
          asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(dst + c * A_LBO), "r"(0) : "memory");
      }
    }
  };
  // (issuer) the nine taps' B tiles of group g -- taps 9 g .. 9 g + 8,
  // consecutive in the packed weights -- into stage g % kTcStages by one
  // bulk copy, completing on the stage's B barrier
  int b_issued = -1, b_waited = -1;  // issuer: last group whose B copy was issued / waited for
  auto fill_b = [&](int g) {
    constexpr uint32_t kBBytes = 9u * N * K * 2u;
    const uint32_t bb = smem_u32(&bbars[g % kTcStages]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(kBBytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sbase + (g % kTcStages) * STAGE + A_BYTES),
                 "l"(Wk + (size_t)(9 * g) * N * K), "r"(kBBytes), "r"(bb)
                 : "memory");
    b_issued = g;
  };

  if (producer) {
    // Each producer refills a stage once the MMAs of the group that read it
    // have completed, waits for its own copies, makes its writes visible to
    // the tensor core's (async) proxy and arrives on the stage's full
    // barrier; it never waits for the issuing thread.
#pragma unroll 1
    for (int g = 0; g < kTcGroups; ++g) {
      if (g >= kTcStages &&
          !mbar_wait_or_stop(&empty[g % kTcStages], (uint32_t)(((g - kTcStages) / kTcStages) & 1), stage_polls,
                             &stop)) {
        fail();
        break;
      }
      fill(g);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[g % kTcStages])) : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else if (issuer) {
    constexpr uint32_t idesc = tc_idesc<N>();
    // the B tiles of the first groups (their stages start free)
    for (int g = 0; g < kTcStages; ++g) fill_b(g);
    int issued = -1;
#pragma unroll 1
    for (int g = 0; g < kTcGroups; ++g) {
      const uint32_t par = (uint32_t)((g / kTcStages) & 1);
      if (!mbar_wait_or_stop(&full[g % kTcStages], par, stage_polls, &stop)) {
        fail();
        break;
      }
      const bool b_ok = mbar_wait(&bbars[g % kTcStages], par, kTcWaitLimit);
      b_waited = g;
      if (!b_ok) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = sbase + (g % kTcStages) * STAGE;
      // one descriptor per operand and group; each MMA adds its offset to
      // the start-address field (address / 16 in the low 14 bits, which
      // cannot carry: shared-memory addresses stay below 256 KB)
      const uint64_t ad = tc_desc(st, A_LBO, 128), bd = tc_desc(st + A_BYTES, B_LBO, 128);
      const uint32_t a_lbo16 = A_LBO >> 4;
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        // tap (dx, dy) = SIGN (j % 3 - 1, j / 3 - 1): output row m reads
        // window row m + LXP + 1 + SIGN (dx + dy LXP)
        const int dx = SIGN * (j % 3 - 1), dy = SIGN * (j / 3 - 1);
        const uint32_t arow = (uint32_t)(LXP + 1 + dx + dy * LXP);
#pragma unroll
        for (int q = 0; q < K / 16; ++q)
          tc_mma(tmem, ad + (arow + (uint32_t)q * 2 * a_lbo16), bd + (uint32_t)((j * B_TAP + q * 2 * B_LBO) >> 4),
                 idesc, (g > 0 || j > 0 || q > 0) ? 1u : 0u);
      }
      tc_commit(&empty[g % kTcStages]);
      issued = g;
      // the stage of group g - 1 takes group g - 1 + S's B tiles once its
      // MMAs (queued ahead of group g's) have completed
      if (g >= 1 && g - 1 + kTcStages < kTcGroups) {
        if (!mbar_wait_or_stop(&empty[(g - 1) % kTcStages], (uint32_t)(((g - 1) / kTcStages) & 1), kTcWaitLimit,
                               &stop)) {
          fail();
          break;
        }
        fill_b(g - 1 + kTcStages);
      }
    }
    // B copies still in flight (after an early exit) land before the CTA ends
    for (int gg = b_waited + 1; gg <= b_issued; ++gg)
      (void)mbar_wait(&bbars[gg % kTcStages], (uint32_t)((gg / kTcStages) & 1), kTcWaitLimit);
    // all MMAs issued so far have completed once the last commit's phase does
    if (issued >= 0) {
      tc_commit(&done_bar);
      if (!mbar_wait(&done_bar, 0u, kTcWaitLimit)) fail();
    }
    last_issued = issued;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int issued = last_issued;
  if (producer && !stop && issued == kTcGroups - 1) {
    float acc[32];
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(32 * w) << 16);
    if constexpr (N == 32) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
          "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
    } else {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr)
          : "memory");
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = __uint_as_float(r[j]);
    if (s_out >= 0) {
      const int so = s_out;
      if constexpr (FWD) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float v = acc[j] + bias[j];
          acc[j] = relu ? fmaxf(v, 0.0f) : v;
        }
        if (yf != nullptr)
#pragma unroll
          for (int j = 0; j < N; j += 4)
            *reinterpret_cast<float4*>(yf + (size_t)so * N + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
      } else if (mask != nullptr) {
        const bf16* mrow = mask + (size_t)so * N;
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (!(__bfloat162float(mrow[j]) > 0.0f)) acc[j] = 0.0f;
      }
      bf16* out = y + (size_t)so * N;
#pragma unroll
      for (int j = 0; j < N; j += 8) {
        uint4 q;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(acc[j], acc[j + 1]), h1 = __floats2bfloat162_rn(acc[j + 2], acc[j + 3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(acc[j + 4], acc[j + 5]), h3 = __floats2bfloat162_rn(acc[j + 6], acc[j + 7]);
        q.x = *reinterpret_cast<uint32_t*>(&h0);
        q.y = *reinterpret_cast<uint32_t*>(&h1);
        q.z = *reinterpret_cast<uint32_t*>(&h2);
        q.w = *reinterpret_cast<uint32_t*>(&h3);
        *reinterpret_cast<uint4*>(out + j) = q;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

// gW[tap, i, o] += sum_s x[s + off(tap), i] gy[s, o]: block (chunk group,
// tap); each warp accumulates 16-site chunks on the tensor cores and adds its
// tile to gW with FP32 atomics (so the sum order, and its last bits, vary).
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv_bwd_weight(const bf16* __restrict__ x, const bf16* __restrict__ gy,
                                                         float* __restrict__ gW, const Geom geo, int chunks_per_warp) {
  __shared__ __align__(32) bf16 sX[4][16 * CI];
  __shared__ __align__(32) float sC[4][CI * CO];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int V = (int)geo.V;
  const int tap = blockIdx.y;
  wm::fragment<wm::accumulator, 16, 16, 16, float> acc[CI / 16][CO / 16];
#pragma unroll
  for (int m = 0; m < CI / 16; ++m)
#pragma unroll
    for (int n = 0; n < CO / 16; ++n) wm::fill_fragment(acc[m][n], 0.0f);
  const int first = (blockIdx.x * 4 + warp) * chunks_per_warp;
  for (int ch = 0; ch < chunks_per_warp; ++ch) {
    const int s0 = (first + ch) * 16;
    if (s0 >= V) break;
    // stage the 16 neighbour rows of x (CI channels each)
    for (int e = lane; e < 16 * (CI / 8); e += 32) {
      const int r = e / (CI / 8), q = e % (CI / 8);
      int c[4];
      site_coords_i(geo.L, s0 + r, c);
      const int nb = tap_site(geo, c, tap, +1);
      *reinterpret_cast<uint4*>(&sX[warp][r * CI + q * 8]) =
          *reinterpret_cast<const uint4*>(x + (size_t)nb * CI + q * 8);
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < CI / 16; ++m) {
      // A[m = i][k = site] = sX[site][i]: column-major, leading dimension CI
      wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::col_major> am;
      wm::load_matrix_sync(am, &sX[warp][m * 16], CI);
#pragma unroll
      for (int n = 0; n < CO / 16; ++n) {
        wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> bm;
        wm::load_matrix_sync(bm, gy + (size_t)s0 * CO + n * 16, CO);
        wm::mma_sync(acc[m][n], am, bm, acc[m][n]);
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int m = 0; m < CI / 16; ++m)
#pragma unroll
    for (int n = 0; n < CO / 16; ++n)
      wm::store_matrix_sync(&sC[warp][(m * 16) * CO + n * 16], acc[m][n], CO, wm::mem_row_major);
  __syncwarp();
  float* dst = gW + (size_t)tap * CI * CO;
  for (int e = lane; e < CI * CO; e += 32) atomicAdd(dst + e, sC[warp][e]);
}

// gb[o] += sum_s gy[s, o]
template <int CO>
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ gy, float* __restrict__ gb, int V) {
  __shared__ float part[256 / CO][CO];
  const int o = threadIdx.x % CO, r = threadIdx.x / CO;
  constexpr int R = 256 / CO;
  float acc = 0.f;
  for (int s = blockIdx.x * R + r; s < V; s += gridDim.x * R) acc += __bfloat162float(gy[(size_t)s * CO + o]);
  part[r][o] = acc;
  __syncthreads();
  if (r == 0) {
    float t = 0.f;
    for (int k = 0; k < R; ++k) t += part[k][o];
    atomicAdd(gb + o, t);
  }
}

// Adam on the FP32 master parameters; bf16 copies of the weights refreshed.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// bf16 weights from the FP32 parameters; the last layer is widened from 8 to
// 16 outputs with zero columns.
// (Wt*: the same weights K-major for the forward tensor-core convolution,
// [tap][out][in])
// Weight tile order of the tensor-core convolutions: for each tap, the N x K
// tile (N rows of K input values) as K/8 chunks of 16 bytes, chunk-major:
// element (tap, n, k) at ((tap K/8 + k/8) N + n) 8 + k % 8.  This is the
// shared-memory order of a B tile, so the three taps of a group arrive by
// one bulk copy.
__device__ __forceinline__ int wtile_index(int tap, int n, int k, int N, int K) {
  return ((tap * (K / 8) + k / 8) * N + n) * 8 + (k & 7);
}

__global__ void k_pack_weights(const float* __restrict__ p, bf16* __restrict__ W1, bf16* __restrict__ W2,
                               bf16* __restrict__ W3, float* __restrict__ b1, float* __restrict__ b2,
                               float* __restrict__ b3, bf16* __restrict__ Wt1, bf16* __restrict__ Wt2,
                               bf16* __restrict__ Wt3) {
  const int n1 = 81 * kFeat * kHid, n2 = 81 * kHid * kHid, n3 = 81 * kHid * kOutPad;
  const int o_b1 = n1, o_W2 = o_b1 + kHid, o_b2 = o_W2 + n2, o_W3 = o_b2 + kHid, o_b3 = o_W3 + 81 * kHid * kOut;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3 + kHid * 2 + kOutPad;
       i += gridDim.x * blockDim.x) {
    if (i < n1) {
      const bf16 v = __float2bfloat16_rn(p[i]);
      const int tap = i / (kFeat * kHid), r = i % (kFeat * kHid), in = r / kHid, o = r % kHid;
      W1[wtile_index(tap, in, o, kFeat, kHid)] = v;
      Wt1[wtile_index(tap, o, in, kHid, kFeat)] = v;
    } else if (i < n1 + n2) {
      const int j = i - n1;
      const bf16 v = __float2bfloat16_rn(p[o_W2 + j]);
      const int tap = j / (kHid * kHid), r = j % (kHid * kHid), in = r / kHid, o = r % kHid;
      W2[wtile_index(tap, in, o, kHid, kHid)] = v;
      Wt2[wtile_index(tap, o, in, kHid, kHid)] = v;
    } else if (i < n1 + n2 + n3) {
      const int j = i - n1 - n2;  // [tap][i][16]
      const int o = j % kOutPad, ti = j / kOutPad;
      const bf16 v = __float2bfloat16_rn(o < kOut ? p[o_W3 + ti * kOut + o] : 0.f);
      const int tap = ti / kHid, in = ti % kHid;
      W3[wtile_index(tap, in, o, kHid, kOutPad)] = v;
      Wt3[wtile_index(tap, o, in, kOutPad, kHid)] = v;
    } else {
      const int j = i - n1 - n2 - n3;
      if (j < kHid)
        b1[j] = p[o_b1 + j];
      else if (j < 2 * kHid)
        b2[j - kHid] = p[o_b2 + j - kHid];
      else
        b3[j - 2 * kHid] = (j - 2 * kHid) < kOut ? p[o_b3 + j - 2 * kHid] : 0.f;
    }
  }
}

// flat gradient (parameter layout) from the padded last-layer gradient
__global__ void k_unpad_grad3(const float* __restrict__ gW3p, const float* __restrict__ gb3p, float* __restrict__ gW3,
                              float* __restrict__ gb3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 81 * kHid * kOut) gW3[i] = gW3p[(i / kOut) * kOutPad + i % kOut];
  if (i < kOut) gb3[i] = gb3p[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned nb128(int n) { return (unsigned)((n + 127) / 128); }

cudaError_t launch_features(int nc, const void* U0, void* x, const Geom& geo, cudaStream_t s) {
  const int V = (int)geo.V;
  if (nc == 9)
    k_features<9><<<nb128(V), 128, 0, s>>>(static_cast<const cx<float>*>(U0), static_cast<bf16*>(x), geo);
  else
    k_features<6><<<nb128(V), 128, 0, s>>>(static_cast<const cx<float>*>(U0), static_cast<bf16*>(x), geo);
  return cudaPeekAtLastError();
}

cudaError_t launch_expmap(int nc, const float* c, int ldc, void* G, int V, cudaStream_t s) {
  if (nc == 9)
    k_expmap<9><<<nb128(V), 128, 0, s>>>(c, ldc, static_cast<cx<float>*>(G), V);
  else
    k_expmap<6><<<nb128(V), 128, 0, s>>>(c, ldc, static_cast<cx<float>*>(G), V);
  return cudaPeekAtLastError();
}

cudaError_t launch_signal(const void* D, int V, float coef, void* gc, cudaStream_t s) {
  k_signal<<<nb128(V), 128, 0, s>>>(static_cast<const cx<float>*>(D), V, coef, static_cast<bf16*>(gc));
  return cudaPeekAtLastError();
}

cudaError_t launch_conv_bwd_weight(int layer, const void* x, const void* gy, float* gW, const Geom& geo,
                                   cudaStream_t s) {
  const int chunks = (int)(geo.V / 16);
  const int cpw = 8;  // 16-site chunks per warp
  dim3 grid((unsigned)((chunks + 4 * cpw - 1) / (4 * cpw)), 81);
  const bf16* xp = static_cast<const bf16*>(x);
  const bf16* gyp = static_cast<const bf16*>(gy);
  if (layer == 1)
    k_conv_bwd_weight<kFeat, kHid><<<grid, 128, 0, s>>>(xp, gyp, gW, geo, cpw);
  else if (layer == 2)
    k_conv_bwd_weight<kHid, kHid><<<grid, 128, 0, s>>>(xp, gyp, gW, geo, cpw);
  else
    k_conv_bwd_weight<kHid, kOutPad><<<grid, 128, 0, s>>>(xp, gyp, gW, geo, cpw);
  return cudaPeekAtLastError();
}

cudaError_t launch_bias_grad(int co, const void* gy, float* gb, int V, cudaStream_t s) {
  const bf16* g = static_cast<const bf16*>(gy);
  if (co == kHid)
    k_bias_grad<kHid><<<120, 256, 0, s>>>(g, gb, V);
  else
    k_bias_grad<kOutPad><<<120, 256, 0, s>>>(g, gb, V);
  return cudaPeekAtLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float c1,
                        float c2, float eps, cudaStream_t s) {
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, c1, c2, eps);
  return cudaPeekAtLastError();
}

cudaError_t launch_pack_weights(const float* p, void* W1, void* W2, void* W3, float* b1, float* b2, float* b3,
                                void* Wt1, void* Wt2, void* Wt3, cudaStream_t s) {
  k_pack_weights<<<256, 256, 0, s>>>(p, static_cast<bf16*>(W1), static_cast<bf16*>(W2), static_cast<bf16*>(W3), b1,
                                     b2, b3, static_cast<bf16*>(Wt1), static_cast<bf16*>(Wt2),
                                     static_cast<bf16*>(Wt3));
  return cudaPeekAtLastError();
}

namespace {
template <int K, int N, int SIGN, bool FWD>
cudaError_t conv_tc_launch(const void* act, const void* Wk, const float* bias, const void* mask, void* y, float* yf,
                           const Geom& geo, bool relu, int* err, cudaStream_t s) {
  // the stages of the longest x extent fix the attribute once; a launch asks
  // for its own extent's stages
  constexpr int smem_max = kTcStages * tc_stage_bytes<K, N>(kMaxL);
  static_assert(smem_max <= 227 * 1024, "the stages fit one CTA's shared memory");
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_conv_tc<K, N, SIGN, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (attr != cudaSuccess) return attr;
  if (geo.L[0] > kMaxL || geo.L[1] > kMaxL) return cudaErrorInvalidValue;
  const int smem = kTcStages * tc_stage_bytes<K, N>(geo.L[0]);
  // 128 rows per CTA over the (z, t) planes padded by a halo in x and y
  const int64_t rows = (int64_t)(geo.L[0] + 2) * (geo.L[1] + 2) * geo.L[2] * geo.L[3];
  const unsigned nb = (unsigned)((rows + 127) / 128);
  k_conv_tc<K, N, SIGN, FWD><<<nb, kTcThreads, smem, s>>>(static_cast<const bf16*>(act), static_cast<const bf16*>(Wk), bias,
                                                    static_cast<const bf16*>(mask), static_cast<bf16*>(y), yf, geo,
                                                    relu, err);
  return cudaPeekAtLastError();
}
}  // namespace

// forward on the tensor cores: layer 1 48 -> 32, 2 32 -> 32 (both ReLU), 3
// 32 -> 16 (8 used, FP32 copy in yf); Wt the K-major weights
cudaError_t launch_conv_fwd_tc(int layer, const void* x, const void* Wt, const float* b, void* y, float* yf,
                               const Geom& geo, int* err, cudaStream_t s) {
  if (layer == 1) return conv_tc_launch<kFeat, kHid, +1, true>(x, Wt, b, nullptr, y, yf, geo, true, err, s);
  if (layer == 2) return conv_tc_launch<kHid, kHid, +1, true>(x, Wt, b, nullptr, y, yf, geo, true, err, s);
  return conv_tc_launch<kHid, kOutPad, +1, true>(x, Wt, b, nullptr, y, yf, geo, false, err, s);
}

// gradient with respect to the input of layer 3 (32 <- 16) or 2 (32 <- 32) on
// the tensor cores, masked by the ReLU of the layer below (a); W in its own
// [tap][in][out] layout, which is K-major for this product
cudaError_t launch_conv_bwd_data_tc(int layer, const void* gy, const void* W, const void* a, void* gx,
                                    const Geom& geo, int* err, cudaStream_t s) {
  if (layer == 3) return conv_tc_launch<kOutPad, kHid, -1, false>(gy, W, nullptr, a, gx, nullptr, geo, false, err, s);
  return conv_tc_launch<kHid, kHid, -1, false>(gy, W, nullptr, a, gx, nullptr, geo, false, err, s);
}

cudaError_t launch_unpad_grad3(const float* gW3p, const float* gb3p, float* gW3, float* gb3, cudaStream_t s) {
  k_unpad_grad3<<<nb128(81 * kHid * kOut), 128, 0, s>>>(gW3p, gb3p, gW3, gb3);
  return cudaPeekAtLastError();
}

}  // namespace warm
}  // namespace lgf
