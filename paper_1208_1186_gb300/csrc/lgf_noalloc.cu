// lgf_functional_noalloc: F and theta of caller-held device links without
// allocating any memory.
//
// Who needs it: a host program that reserves the GPU's memory for its own
// pool and forbids the libraries it loads from calling cudaMalloc (the call
// would fail, or fragment and unbalance that pool), and monitoring code that
// must read the gauge functional of a running job without changing that
// job's memory footprint.  Such callers pass the links and the output in
// memory they already own; the only other memory the computation needs -- one
// FP64 partial sum pair per thread block -- lives in a fixed-size array
// compiled into this library.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (kNoallocMaxBlocks * 16 bytes = 256 KiB) until the process
// exits.  All calls share it and it keeps the last call's contents; each call
// writes every slot it later reads, so nothing needs clearing.  Calls whose
// work overlaps on the GPU (different streams, or different host threads
// without ordering between them) race on the array and give wrong results:
// order them on one stream or synchronise between them.
//
// Host code never dereferences the array's name: on the host it is only a
// stand-in symbol.  The device address comes from cudaGetSymbolAddress with
// the caller's device current.  A call whose stream is not capturing looks it
// up again every time (a few microseconds of host work), so the address
// always belongs to the current context, also after cudaDeviceReset or when
// the caller runs in a context of its own; the result is remembered per
// device for calls made during stream capture, which reuse the address of the
// last uncaptured call on that device.  So make one uncaptured call, in the
// context the capture will use, before capture begins.
#include <mutex>
#include <string>

#include "../../include/lgf.h"
#include "lgf_kernels.cuh"

namespace lgf {

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 16384;  // 256 KiB of partials
constexpr int64_t kNoallocMaxSites = (int64_t)kNoallocMaxBlocks * kNoallocThreads;  // 4,194,304
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_partials[kNoallocMaxBlocks];

std::mutex g_symbol_mutex;
double2* g_symbol_addr[kMaxDevices] = {};

__device__ __forceinline__ void block_sum2_na(double& a, double& b) {
  __shared__ double sa[32], sb[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    a = l < nw ? sa[l] : 0.0;
    b = l < nw ? sb[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

// Per-site Re Tr U and Tr Delta Delta^dagger, summed per block into
// partial[blockIdx.x]; the gradient itself is not stored.
template <class T, int NC>
__global__ void __launch_bounds__(kNoallocThreads) k_functional_partials(const cx<T>* __restrict__ U,
                                                                       double2* __restrict__ partial,
                                                                       const Geom geo) {
  const int64_t V = geo.V;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double fsum = 0.0, tsum = 0.0;
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
      fsum += (double)own.e[0][0].re + (double)own.e[1][1].re + (double)own.e[2][2].re;
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
    const double di0 = a0 - tr, di1 = a1 - tr, di2 = -(di0 + di1);
    tsum = 2.0 * ((double)norm2(cvt<double>(d01)) + (double)norm2(cvt<double>(d02)) +
                  (double)norm2(cvt<double>(d12))) +
           di0 * di0 + di1 * di1 + di2 * di2;
  }
  block_sum2_na(fsum, tsum);
  if (threadIdx.x == 0) partial[blockIdx.x] = make_double2(fsum, tsum);
}

// Fixed-order sum of the n partials -> out[0] = F, out[1] = theta.
__global__ void __launch_bounds__(1024) k_functional_final(const double2* __restrict__ partial, int n,
                                                           double* __restrict__ out, double normF,
                                                           double normT) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 p = partial[i];
    a += p.x;
    b += p.y;
  }
  block_sum2_na(a, b);
  if (threadIdx.x == 0) {
    out[0] = a * normF;
    out[1] = b * normT;
  }
}

// Device address of the partials array in the current context.  Outside
// stream capture it is looked up on every call and remembered per device;
// during capture the remembered address is used (*out stays null if there is
// none yet).
cudaError_t partials_address(cudaStream_t s, double2** out) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_symbol_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_symbol_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_symbol_addr[dev];
  return cudaSuccess;
}

int noalloc_fail(int code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

}  // namespace

}  // namespace lgf

using namespace lgf;

extern "C" int lgf_functional_noalloc(const void* links, int Lx, int Ly, int Lz, int Lt, int dtype, double* out,
                                      void* stream) {
  const int Ls[4] = {Lx, Ly, Lz, Lt};
  Geom geo{};
  int64_t V = 1;
  for (int a = 0; a < 4; ++a) {
    if (Ls[a] < 2 || Ls[a] > kMaxL)
      return noalloc_fail(LGF_ERR_ARG, "lgf_functional_noalloc: each lattice extent must be in [2, 64]");
    geo.L[a] = Ls[a];
    geo.stride[a] = V;
    V *= Ls[a];
  }
  geo.V = V;
  geom_init_rcp(geo);
  if (V > kNoallocMaxSites)
    return noalloc_fail(LGF_ERR_ARG, "lgf_functional_noalloc: the lattice has " + std::to_string(V) +
                                         " sites; this entry point supports at most " +
                                         std::to_string(kNoallocMaxSites) + " (its fixed scratch holds " +
                                         std::to_string(kNoallocMaxBlocks) + " block sums)");
  if (dtype < LGF_F64 || dtype > LGF_F64_R12) return noalloc_fail(LGF_ERR_ARG, "lgf_functional_noalloc: unknown dtype");
  if (links == nullptr || out == nullptr)
    return noalloc_fail(LGF_ERR_ARG, "lgf_functional_noalloc: links and out must be device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double2* partial = nullptr;
  cudaError_t e = partials_address(s, &partial);
  if (e != cudaSuccess)
    return noalloc_fail(LGF_ERR_CUDA, std::string("lgf_functional_noalloc: scratch address lookup: ") +
                                          cudaGetErrorString(e));
  if (partial == nullptr)
    return noalloc_fail(LGF_ERR_ARG,
                        "lgf_functional_noalloc: called during stream capture before any uncaptured call on this "
                        "device (the scratch array's address is looked up outside capture)");
  const int nb = (int)((V + kNoallocThreads - 1) / kNoallocThreads);
  const bool f64 = (dtype == LGF_F64 || dtype == LGF_F64_R12);
  const bool r12 = (dtype == LGF_F32_R12 || dtype == LGF_F64_R12);
  if (f64 && !r12)
    k_functional_partials<double, 9><<<nb, kNoallocThreads, 0, s>>>(static_cast<const cx<double>*>(links), partial, geo);
  else if (f64)
    k_functional_partials<double, 6><<<nb, kNoallocThreads, 0, s>>>(static_cast<const cx<double>*>(links), partial, geo);
  else if (!r12)
    k_functional_partials<float, 9><<<nb, kNoallocThreads, 0, s>>>(static_cast<const cx<float>*>(links), partial, geo);
  else
    k_functional_partials<float, 6><<<nb, kNoallocThreads, 0, s>>>(static_cast<const cx<float>*>(links), partial, geo);
  k_functional_final<<<1, 1024, 0, s>>>(partial, nb, out, 1.0 / (12.0 * (double)V), 1.0 / (3.0 * (double)V));
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(LGF_ERR_CUDA, std::string("lgf_functional_noalloc: launch: ") + cudaGetErrorString(e));
  return LGF_OK;
}
