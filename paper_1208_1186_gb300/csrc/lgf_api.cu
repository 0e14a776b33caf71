// C ABI of liblgf (declared in include/lgf.h): handle management, device
// buffers, and the host-side queueing of gauge-fixing iterations.
//
// One iteration (Sec. 1 of the paper: steepest descent with Fourier
// acceleration; Sec. 2.2: one thread per site, 2D plus 2D FFT) is the kernel
// chain
//   gradient -> reduce -> fft_xy(fwd) -> fft_zt(fwd, scale, inv)
//            -> fft_xy(inv) -> build_g -> update [-> accumulate G]
// on the handle's stream.  The reduce kernel decides on the device whether
// the update of its iteration is applied (theta < tol or max_iter reached
// stop the queue); every later kernel reads that decision first, so lgf_fix
// queues LGF_CHECK_EVERY iterations between host synchronisations and still
// stops at exactly the first iteration with theta < tol.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lgf.h"
#include "fft_reg.cuh"
#include "lgf_kernels.cuh"

using namespace lgf;

namespace {

thread_local std::string g_last_create_error;

struct Allocator {
  lgf_alloc_fn alloc = nullptr;
  lgf_free_fn free_fn = nullptr;
  void* user = nullptr;
};
Allocator g_alloc;

// Buffers of one working precision: links, packed gradient, gauge step,
// twiddle factors.
struct Engine {
  int prec = 8;  // bytes per real: 8 (FP64) or 4 (FP32)
  int nc = 9;    // complex entries stored per matrix
  void* U = nullptr;
  void* D = nullptr;
  void* g = nullptr;
  void* tw = nullptr;
  FftGeom fg{};  // FFT tiling for this precision (plane pipeline)
  bool axis = false;     // per-axis register FFT passes apply to this lattice
  bool plane = false;    // three-pass register plane pipeline applies
  int tuned = 0;         // pipeline chosen by lgf_autotune or the tuning cache (0: none)
  int zt_bx = 0;         // plane pipeline: x-run width of the z-t tiles (0: default)
  int zt_ro = 0;         // plane pipeline: radix order of the z and t transforms
  bool grep = false;     // FP32 engine: gauge representation (U holds the loaded links, G is updated)
  void* kfac = nullptr;  // axis pipeline, FP64: p2_max/(V p2(k)) per site, digit-reversed order
  float* s2p = nullptr;  // FP32: [3][4][kMaxL] 4 sin^2(pi k/L) at the digit-reversed positions of radix order 0, 1
                         // and at the tile slots of order 2 (the pair split)
  float c_over_V = 0.f;  // p2_max / V
  size_t cbytes() const { return 2 * (size_t)prec; }
};

// FFT schedule of one (precision, lattice shape): the pipeline and, for the
// plane pipeline, the z-t tile width and radix order (lgf_autotune); kept for
// the process and optionally in a JSON file (lgf_tune_save / lgf_tune_load)
struct TuneEntry {
  int pipeline = 0;
  int zt_bx = 0;
  int zt_ro = 0;
  double ms = 0.0;  // per Fourier acceleration, as timed by the autotuner
};
using TuneKey = std::tuple<int, int, int, int, int>;  // (bytes per real, Lx, Ly, Lz, Lt)
std::mutex g_tune_mutex;
std::map<TuneKey, TuneEntry> g_tune_cache;
bool g_tune_apply_at_create = false;  // set once a cache file has been loaded
std::once_flag g_tune_env_once;

}  // namespace

void lgf::set_global_error(const std::string& msg) { g_last_create_error = msg; }

struct lgf_ctx {
  int L[4] = {0, 0, 0, 0};
  int64_t V = 0;
  int dtype = 0;
  bool mixed = false;  // FP32 bulk + FP64 tail
  int device = 0;
  cudaStream_t stream = nullptr;
  double alpha = 0.08;
  int check_every = 32;
  double tail_theta = 1e-12;
  long long tail_max32 = -1;
  bool reunit_fp64 = false;   // FP32 storage: reunitarise g in FP64 arithmetic
  int fft_pipeline = 0;       // 0 auto, 1 Stockham planes, 2 axis passes, 3 register planes
  bool explicit_fp32 = false; // FP32 engine: update the links in place instead of G (from the next load)
  int exp_order = 1;          // g from 1 + alpha/2 Delta~ (1) or from its exact exponential (0)
  bool track_g = false;       // FP64 handles, from the next load: accumulate G <- g G (LGF_TRACK_G)
  bool g64_track = false;     // ... in effect since the last load (G holds e64.nc FP64 planes)
  bool g_valid = false;       // G (with the tail's Gh, Gl and eta) describes the current links
  int tail_mode = 0;          // defect-correction tail when the FP32 phase reached 1e-8, with links in
                              // double-float (0) or FP64 (2); 1: plain FP64
  bool defect = false;        // the FP64 engine runs the defect-correction tail
  bool df = false;            // ... on the double-float links in Udf (converted back at the end)
  void* Udf = nullptr;        // tail links in double-float: 36 V complex hi, then 36 V complex lo
  void* eta = nullptr;        // the tail's gauge transformation 1 + eta: 9 V complex hi, then 9 V lo
  void* tbase = nullptr;      // the tail gradient's fixed part: Delta(Udf) (4 V complex), F terms (V float pairs)

  Geom geo{};
  Engine e64, e32;
  Engine* cur = nullptr;     // engine that holds the current links
  void* G = nullptr;         // mixed: accumulated gauge transformation (e32 storage)
  double* Uorig = nullptr;   // mixed: FP64 SoA copy of the loaded links (9 planes)
  double* sin2 = nullptr;    // [4][kMaxL] 4 sin^2(pi k / L)
  double2* partial = nullptr;
  int nblk = 0;
  DevState* st = nullptr;    // device
  DevState* st_host = nullptr;  // pinned mirror
  double* hist = nullptr;
  int hist_cap = 0;
  int hist_n = 0;
  double* staging = nullptr;  // device FP64 AoS link buffer (V*72 doubles), lazily
  size_t staging_bytes = 0;
  double* staging_out = nullptr;  // second such buffer, for the results of lgf_fix_stream
  bool loaded = false;
  long long launches = 0;
  long long total_updates = 0;
  // device-side iteration loops (lgf_fix without profiling): one CUDA graph
  // per loop kind, a while node around one captured iteration
  struct DevLoop {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long cond = 0;
    long long launches = 0;  // kernels per iteration
  };
  DevLoop loops[4];
  cudaStream_t cap_stream = nullptr;  // capture stream of the loop bodies
  int last_n32 = 0, last_n64 = 0;  // split of the last lgf_fix
  std::string err;
  // per-kernel timing (lgf_profile): an event before and after each launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;  // kernel kind of event pair i (events 2i, 2i+1)
  double prof_ms[LGF_NUM_KERNELS] = {};
  long long prof_n[LGF_NUM_KERNELS] = {};
  struct Alloc {
    void* p;
    size_t n;
  };
  std::vector<Alloc> allocs;
};

namespace {

// lgf_fix without profiling runs each phase as one device-side graph loop
constexpr bool kDeviceLoops = true;

int fail(lgf_handle h, int code, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_last_create_error = msg;
  return code;
}

int cuda_fail(lgf_handle h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(h, LGF_ERR_CUDA, m);
}

#define LGF_CUDA(h, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

// event slot for the next profiled launch (grows the pool on demand)
cudaError_t prof_begin(lgf_handle h, int kind) {
  const size_t i = h->ev_kind.size();
  while (h->ev_pool.size() < 2 * i + 2) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    h->ev_pool.push_back(ev);
  }
  h->ev_kind.push_back(kind);
  return cudaEventRecord(h->ev_pool[2 * i], h->stream);
}

cudaError_t prof_end(lgf_handle h) {
  return cudaEventRecord(h->ev_pool[2 * (h->ev_kind.size() - 1) + 1], h->stream);
}

// Launch one kernel of the given kind, counting it and, when profiling,
// bracketing it with events on the handle's stream.
#define LGF_LAUNCH(h, kind, call)                             \
  do {                                                        \
    if ((h)->profiling) LGF_CUDA(h, prof_begin((h), (kind))); \
    LGF_CUDA(h, call);                                        \
    if ((h)->profiling) LGF_CUDA(h, prof_end(h));             \
    (h)->launches += 1;                                       \
  } while (0)

void* dev_alloc(lgf_handle h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (g_alloc.alloc) {
    p = g_alloc.alloc(bytes, h->device, (void*)h->stream, g_alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    p = nullptr;
  }
  if (p) h->allocs.push_back({p, bytes});
  return p;
}

void dev_free_all(lgf_handle h) {
  for (auto& a : h->allocs) {
    if (g_alloc.free_fn)
      g_alloc.free_fn(a.p, a.n, h->device, (void*)h->stream, g_alloc.user);
    else
      cudaFree(a.p);
  }
  h->allocs.clear();
}

int alloc_engine(lgf_handle h, Engine& e) {
  const int64_t V = h->V;
  e.U = dev_alloc(h, (size_t)4 * e.nc * V * e.cbytes());
  e.D = dev_alloc(h, (size_t)4 * V * e.cbytes());
  e.g = dev_alloc(h, (size_t)9 * V * e.cbytes());
  e.tw = dev_alloc(h, (size_t)4 * kMaxL * e.cbytes());
  if (!e.U || !e.D || !e.g || !e.tw) return fail(h, LGF_ERR_OOM, "device allocation failed");
  // twiddle factors e^{-2 pi i m / L} per axis, computed in long double
  std::vector<double> tw64(8 * kMaxL, 0.0);
  std::vector<float> tw32(8 * kMaxL, 0.0f);
  for (int a = 0; a < 4; ++a) {
    const int L = h->L[a];
    for (int m = 0; m < L; ++m) {
      const long double ang = 2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)L;
      const double c = (double)cosl(ang), s = (double)-sinl(ang);
      tw64[2 * (a * kMaxL + m)] = c;
      tw64[2 * (a * kMaxL + m) + 1] = s;
      tw32[2 * (a * kMaxL + m)] = (float)c;
      tw32[2 * (a * kMaxL + m) + 1] = (float)s;
    }
  }
  if (e.prec == 8)
    LGF_CUDA(h, cudaMemcpy(e.tw, tw64.data(), tw64.size() * sizeof(double), cudaMemcpyHostToDevice));
  else
    LGF_CUDA(h, cudaMemcpy(e.tw, tw32.data(), tw32.size() * sizeof(float), cudaMemcpyHostToDevice));
  e.axis = true;
  for (int a = 0; a < 4; ++a) e.axis = e.axis && axis_pass_supported(e.prec, h->L[a]);
  e.plane = plane_pipeline_supported(e.prec, h->L[0], h->L[1], h->L[2], h->L[3]);
  if (e.axis || e.plane) {
    // acceleration factor at every position the forward passes leave a mode:
    // position p along an axis holds frequency digit_rev(L, p)
    std::vector<double> s2[4];
    std::vector<float> s2f(3 * 4 * kMaxL, 0.0f);
    double p2max = 0.0;
    for (int a = 0; a < 4; ++a) {
      const int L = h->L[a];
      s2[a].resize(L);
      double m = 0.0;
      for (int p = 0; p < L; ++p) {
        const long double sk =
            sinl(3.14159265358979323846264338327950288L * (long double)regfft::digit_rev(L, p) / (long double)L);
        s2[a][p] = (double)(4.0L * sk * sk);
        s2f[a * kMaxL + p] = (float)s2[a][p];
        m = s2[a][p] > m ? s2[a][p] : m;
        // the same at the positions of radix order 1
        const long double sk1 = sinl(3.14159265358979323846264338327950288L *
                                     (long double)regfft::digit_rev(L, p, 1) / (long double)L);
        s2f[4 * kMaxL + a * kMaxL + p] = (float)(4.0L * sk1 * sk1);
        // the pair split: slot 2 q + half holds frequency pair_freq(L, q, half)
        if (regfft::pair_supported(L)) {
          const long double sk2 = sinl(3.14159265358979323846264338327950288L *
                                       (long double)regfft::pair_freq(L, p >> 1, p & 1) / (long double)L);
          s2f[2 * 4 * kMaxL + a * kMaxL + p] = (float)(4.0L * sk2 * sk2);
        }
      }
      p2max += m;
    }
    e.c_over_V = (float)(p2max / (double)V);
    if (e.prec == 4) {
      e.s2p = static_cast<float*>(dev_alloc(h, s2f.size() * sizeof(float)));
      if (!e.s2p) return fail(h, LGF_ERR_OOM, "device allocation failed");
      LGF_CUDA(h, cudaMemcpy(e.s2p, s2f.data(), s2f.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      e.kfac = dev_alloc(h, (size_t)V * e.prec);
      if (!e.kfac) return fail(h, LGF_ERR_OOM, "device allocation failed");
      std::vector<double> k64(V);
      int64_t s = 0;
      for (int t = 0; t < h->L[3]; ++t)
        for (int z = 0; z < h->L[2]; ++z)
          for (int y = 0; y < h->L[1]; ++y)
            for (int x = 0; x < h->L[0]; ++x, ++s)
              k64[s] = (x | y | z | t) ? p2max / ((s2[0][x] + s2[1][y] + s2[2][z] + s2[3][t]) * (double)V) : 0.0;
      LGF_CUDA(h, cudaMemcpy(e.kfac, k64.data(), (size_t)V * 8, cudaMemcpyHostToDevice));
    }
  }
  return LGF_OK;
}

int tune_load_file(const char* path, int* n_out);

// A cached schedule (from a loaded tuning file, or tuned in this process
// after one was loaded) for engine e's precision and shape, if it applies.
void apply_cached_schedule(lgf_handle h, Engine& e) {
  std::call_once(g_tune_env_once, [] {
    const char* path = getenv("LGF_TUNE_CACHE");
    if (path && *path) tune_load_file(path, nullptr);
  });
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (!g_tune_apply_at_create) return;
  auto it = g_tune_cache.find(std::make_tuple(e.prec, h->L[0], h->L[1], h->L[2], h->L[3]));
  if (it == g_tune_cache.end()) return;
  const TuneEntry& t = it->second;
  if ((t.pipeline == 2 && !e.axis) || (t.pipeline == 3 && !e.plane)) return;
  e.tuned = t.pipeline;
  e.zt_bx = t.zt_bx;
  e.zt_ro = t.zt_ro;
}

int ensure_staging(lgf_handle h) {
  const size_t need = (size_t)h->V * 72 * sizeof(double);
  if (h->staging && h->staging_bytes >= need) return LGF_OK;
  h->staging = static_cast<double*>(dev_alloc(h, need));
  if (!h->staging) return fail(h, LGF_ERR_OOM, "device allocation of the link staging buffer failed");
  h->staging_bytes = need;
  return LGF_OK;
}

int sync_state(lgf_handle h) {
  LGF_CUDA(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

int reset_state(lgf_handle h, double tol, int max_iter, bool with_hist, bool stall = false,
                bool use_cond = false, unsigned long long cond = 0) {
  DevState s{};
  s.stall = stall ? 1 : 0;
  s.use_cond = use_cond ? 1 : 0;
  s.cond = cond;
  s.F = 0.0;
  s.theta = 0.0;
  s.done = 0;
  s.iters = 0;
  s.nonfinite = 0;
  s.max_iter = max_iter;
  s.tol = tol;
  s.hist = with_hist ? h->hist : nullptr;
  s.hist_cap = with_hist ? h->hist_cap : 0;
  *h->st_host = s;
  LGF_CUDA(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  return LGF_OK;
}

// FFT pipeline for engine e: the register plane pipeline (3 passes) where
// its shapes are instantiated, else the per-axis register passes (7), else
// the shared-memory Stockham plane kernels; LGF_FFT_PIPELINE can force one
// (falling back to Stockham where the forced one does not apply).
int pick_pipeline(lgf_handle h, const Engine& e) {
  if (h->fft_pipeline == 0 && e.tuned != 0) return e.tuned;
  switch (h->fft_pipeline) {
    case 1: return 1;
    case 2: return e.axis ? 2 : 1;
    case 3: return e.plane ? 3 : 1;
    default: return e.plane ? 3 : (e.axis ? 2 : 1);
  }
}

// Fourier acceleration of the packed gradient in e.D (forward 4D FFT, times
// p2_max/(V p2), inverse).
int queue_accelerate(lgf_handle h, Engine& e, const DevState* st) {
  cudaStream_t s = h->stream;
  const int pipe = pick_pipeline(h, e);
  if (pipe == 3) {
    const int* L = h->L;
    LGF_LAUNCH(h, LGF_K_FFT_XY, launch_plane_xy(e.prec, L[0], e.D, h->V, L[2], L[3], 0, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_ZT, launch_plane_zt(e.prec, L[0], L[1], L[2], L[3], e.D, e.kfac, e.s2p, e.c_over_V,
                                                e.zt_bx, e.zt_ro, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_XY, launch_plane_xy(e.prec, L[0], e.D, h->V, L[2], L[3], 1, st, s));
  } else if (pipe == 2) {
    const int64_t V = h->V;
    const int64_t Sy = h->L[0], Sz = (int64_t)h->L[0] * h->L[1];
    LGF_LAUNCH(h, LGF_K_FFT_AXIS, launch_xpass(e.prec, h->L[0], e.D, V, 0, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_AXIS, launch_strided(e.prec, h->L[1], e.D, V, Sy, 0, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_AXIS, launch_strided(e.prec, h->L[2], e.D, V, Sz, 0, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_T, launch_tpass(e.prec, h->L[3], e.D, V, h->L[0], h->L[1], e.kfac, e.s2p, e.c_over_V,
                                            st, s));
    LGF_LAUNCH(h, LGF_K_FFT_AXIS, launch_strided(e.prec, h->L[2], e.D, V, Sz, 1, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_AXIS, launch_strided(e.prec, h->L[1], e.D, V, Sy, 1, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_AXIS, launch_xpass(e.prec, h->L[0], e.D, V, 1, st, s));
  } else {
    LGF_LAUNCH(h, LGF_K_FFT_XY, launch_fft_xy(e.prec, e.D, e.fg, e.tw, 0, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_ZT, launch_fft_zt(e.prec, e.D, e.fg, e.tw, h->sin2, st, s));
    LGF_LAUNCH(h, LGF_K_FFT_XY, launch_fft_xy(e.prec, e.D, e.fg, e.tw, 1, st, s));
  }
  return LGF_OK;
}

// FP64 tail start of a mixed handle after its FP32 phase: the gauge G
// reunitarised (in double-float for the double-float tail, else in FP64),
// then the links rebuilt from the loaded input as G U_loaded G^dagger.  The
// defect-correction tail (theta < 1e-8 at the hand-over, tail modes 0 and 2)
// and, in mode 0, its double-float form are chosen here; that form also
// clears the tail's gauge transformation and forms its gradient's fixed part.
int queue_tail_start(lgf_handle h) {
  const int64_t V = h->V;
  h->defect = h->tail_mode != 1 && h->st_host->theta < 1e-8;
  h->df = h->defect && h->tail_mode == 0;
  if (h->df) {
    // each buffer on its own, so that a failed allocation is retried by the next tail start
    if (!h->Udf) h->Udf = dev_alloc(h, (size_t)2 * 36 * V * sizeof(float) * 2);
    if (!h->eta) h->eta = dev_alloc(h, (size_t)18 * V * sizeof(float) * 2);
    if (!h->tbase) h->tbase = dev_alloc(h, (size_t)5 * V * sizeof(float) * 2);
    if (!h->Udf || !h->eta || !h->tbase) {
      h->df = false;
      return fail(h, LGF_ERR_OOM, "device allocation of the double-float tail failed");
    }
    // e64.g (9 FP64 complex planes) holds Gh and Gl (2 x 9 FP32 complex planes)
    LGF_LAUNCH(h, LGF_K_OTHER, launch_promote_df(h->G, h->e64.g, V, h->stream));
    LGF_LAUNCH(h, LGF_K_UPDATE, launch_tail_start_df(h->Uorig, h->e64.g, h->Udf, h->geo, h->stream));
    LGF_CUDA(h, cudaMemsetAsync(h->eta, 0, (size_t)18 * V * sizeof(float) * 2, h->stream));
    LGF_LAUNCH(h, LGF_K_OTHER, launch_tail_base(h->Udf, h->tbase, h->geo, h->stream));
  } else {
    h->g_valid = false;  // the FP64 tails update the links without tracking their gauge transformation
    LGF_LAUNCH(h, LGF_K_OTHER, launch_promote_gauge(4, h->e32.nc, h->G, h->e64.g, V, h->stream));
    LGF_CUDA(h, cudaMemcpyAsync(h->e64.U, h->Uorig, (size_t)4 * 9 * V * 16, cudaMemcpyDeviceToDevice, h->stream));
    LGF_LAUNCH(h, LGF_K_UPDATE, launch_update(8, 9, h->e64.U, h->e64.g, h->geo, nullptr, h->stream));
  }
  h->cur = &h->e64;
  return LGF_OK;
}

// After a double-float tail the handle's links stay in that form, U' = (1 +
// eta) Udf (1 + eta(x+mu))^dag (h->df): later fixes and iterations continue
// on them, lgf_functional takes their gradient and lgf_store_links writes
// FP64 from them directly.  Calls that need the links as FP64 planes apply
// eta to Udf and convert here first.
int materialize_df(lgf_handle h) {
  if (!h->df || h->cur != &h->e64) return LGF_OK;
  h->g_valid = false;  // later iterations run on the FP64 links
  LGF_LAUNCH(h, LGF_K_OTHER, launch_tail_apply_eta(h->Udf, h->eta, h->geo, h->stream));
  LGF_LAUNCH(h, LGF_K_OTHER, launch_df_to_fp64(h->Udf, h->e64.U, h->V, h->stream));
  h->df = false;
  return LGF_OK;
}

// Gradient (+ F/theta reduction) of the engine's current links.
int queue_gradient(lgf_handle h, Engine& e, int mode) {
  if (&e == &h->e64 && h->df)
    LGF_LAUNCH(h, LGF_K_GRADIENT,
               launch_gradient_tail_eta(h->Udf, h->eta, h->tbase, h->e32.D, h->partial, h->geo, h->st, mode,
                                        h->stream));
  else if (e.grep)
    LGF_LAUNCH(h, LGF_K_GRADIENT,
               launch_gradient_grep(e.nc, e.U, h->G, e.D, h->partial, h->geo, h->st, mode, h->stream));
  else
    LGF_LAUNCH(h, LGF_K_GRADIENT, launch_gradient(e.prec, e.nc, e.U, e.D, h->partial, h->geo, h->st, mode, h->stream));
  return LGF_OK;
}

// One full iteration on engine e, with the stop logic of an iteration queue.
// Gauge representation: gradient, acceleration, G <- g G.  Otherwise:
// gradient, acceleration, g, link update, and on the FP32 engine of a mixed
// handle G <- g G as well, so that the FP32 links always equal
// G U_loaded G^dagger up to FP32 rounding.
int queue_iteration(lgf_handle h, Engine& e) {
  cudaStream_t s = h->stream;
  if (h->defect && h->df && &e == &h->e64) {
    // defect-correction tail on the double-float links of the tail start in
    // gauge representation; FP32 acceleration and step on eta
    Engine& f = h->e32;
    LGF_LAUNCH(h, LGF_K_GRADIENT,
               launch_gradient_tail_eta(h->Udf, h->eta, h->tbase, f.D, h->partial, h->geo, h->st, 1, s));
    if (pick_pipeline(h, f) == 3 && plane_xyinv_eta_supported(h->L[0])) {
      // forward x-y, z-t, then the inverse x-y pass fused with the eta step
      const int* L = h->L;
      LGF_LAUNCH(h, LGF_K_FFT_XY, launch_plane_xy(f.prec, L[0], f.D, h->V, L[2], L[3], 0, h->st, s));
      LGF_LAUNCH(h, LGF_K_FFT_ZT,
                 launch_plane_zt(f.prec, L[0], L[1], L[2], L[3], f.D, f.kfac, f.s2p, f.c_over_V, f.zt_bx, f.zt_ro,
                                 h->st, s));
      LGF_LAUNCH(h, LGF_K_XY_GSTEP,
                 launch_plane_xyinv_eta(L[0], f.D, h->eta, h->V, L[2], L[3], 0.5 * h->alpha, h->st, s));
      return LGF_OK;
    }
    int rc = queue_accelerate(h, f, h->st);
    if (rc) return rc;
    LGF_LAUNCH(h, LGF_K_UPDATE, launch_tail_eta_step(f.D, h->eta, h->V, 0.5 * h->alpha, h->st, s));
    return LGF_OK;
  }
  if (h->defect && &e == &h->e64) {
    // defect-correction tail: FP64 links, FP32 acceleration and step
    Engine& f = h->e32;
    LGF_LAUNCH(h, LGF_K_GRADIENT, launch_gradient_tail(e.U, f.D, h->partial, h->geo, h->st, 1, s));
    int rc = queue_accelerate(h, f, h->st);
    if (rc) return rc;
    LGF_LAUNCH(h, LGF_K_BUILD_G, launch_tail_step(f.D, f.g, h->V, 0.5 * h->alpha, h->st, s));
    LGF_LAUNCH(h, LGF_K_UPDATE, launch_tail_update(e.U, f.g, h->geo, h->st, s));
    return LGF_OK;
  }
  int rc = queue_gradient(h, e, 1);
  if (rc) return rc;
  const bool exact = h->exp_order == 0;
  if (e.grep && !exact && pick_pipeline(h, e) == 3 && plane_xyinv_gstep_supported(e.prec, h->L[0])) {
    // forward x-y, z-t, then the inverse x-y fused with G <- g G
    const int* L = h->L;
    LGF_LAUNCH(h, LGF_K_FFT_XY, launch_plane_xy(e.prec, L[0], e.D, h->V, L[2], L[3], 0, h->st, s));
    LGF_LAUNCH(h, LGF_K_FFT_ZT,
               launch_plane_zt(e.prec, L[0], L[1], L[2], L[3], e.D, e.kfac, e.s2p, e.c_over_V, e.zt_bx, e.zt_ro,
                               h->st, s));
    LGF_LAUNCH(h, LGF_K_XY_GSTEP, launch_plane_xyinv_gstep(L[0], e.nc, e.D, h->G, h->V, L[2], L[3], 0.5 * h->alpha,
                                                           h->reunit_fp64, h->st, s));
    return LGF_OK;
  }
  rc = queue_accelerate(h, e, h->st);
  if (rc) return rc;
  if (e.grep) {
    LGF_LAUNCH(h, LGF_K_BUILD_G,
               launch_gstep(e.nc, e.D, h->G, nullptr, h->V, 0.5 * h->alpha, h->reunit_fp64, exact, h->st, s));
    return LGF_OK;
  }
  LGF_LAUNCH(h, LGF_K_BUILD_G,
             launch_build_g(e.prec, e.nc, e.D, e.g, h->V, 0.5 * h->alpha, h->reunit_fp64, exact, h->st, s));
  LGF_LAUNCH(h, LGF_K_UPDATE, launch_update(e.prec, e.nc, e.U, e.g, h->geo, h->st, s));
  if ((h->mixed && &e == &h->e32) || (!h->mixed && h->g64_track))
    LGF_LAUNCH(h, LGF_K_ACCUMULATE, launch_accumulate(e.prec, e.nc, h->G, e.g, h->V, h->st, s));
  return LGF_OK;
}

// Device-side loops.  Kind 0: an iteration of the FP32 engine (or of a plain
// FP32/FP64 handle's engine); 1: the double-float defect tail; 2: the FP64
// defect tail; 3: the plain FP64 iteration of a mixed handle's tail.
int loop_kind(lgf_handle h, const Engine& e) {
  if (&e == &h->e32 || !h->mixed) return 0;
  if (h->defect) return h->df ? 1 : 2;
  return 3;
}

void drop_loops(lgf_handle h) {
  for (auto& l : h->loops) {
    if (l.exec) cudaGraphExecDestroy(l.exec);
    if (l.graph) cudaGraphDestroy(l.graph);
    l = lgf_ctx::DevLoop{};
  }
}

// A graph holding one conditional while node whose body is one captured
// iteration of engine e.  The gradient kernel's stop decision sets the
// condition (lgf_reduce.cuh): the loop ends once the queue is done, which
// happens at the latest when max_iter updates have been applied.
int build_loop(lgf_handle h, Engine& e, lgf_ctx::DevLoop& l) {
  if (!h->cap_stream) LGF_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  LGF_CUDA(h, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNodeParams p = {};
  cudaGraphNode_t node = nullptr;
  cudaError_t err = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (err == cudaSuccess) {
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    err = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
  }
  if (err != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(h, LGF_ERR_CUDA, std::string("device loop: ") + cudaGetErrorString(err));
  }
  cudaGraph_t body = p.conditional.phGraph_out[0];
  cudaStream_t saved = h->stream;
  h->stream = h->cap_stream;
  const long long l0 = h->launches;
  int rc = LGF_OK;
  err = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    rc = queue_iteration(h, e);
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &out);
    if (!rc && e2 != cudaSuccess) err = e2;
  }
  l.launches = h->launches - l0;
  h->launches = l0;
  h->stream = saved;
  if (!rc && err == cudaSuccess) err = cudaGraphInstantiate(&l.exec, g, 0);
  if (rc || err != cudaSuccess) {
    if (l.exec) cudaGraphExecDestroy(l.exec);
    l.exec = nullptr;
    cudaGraphDestroy(g);
    return rc ? rc : fail(h, LGF_ERR_CUDA, std::string("device loop: ") + cudaGetErrorString(err));
  }
  l.graph = g;
  l.cond = cond;
  return LGF_OK;
}

// Run engine e until theta < tol, max_iter updates, or (if stall_check) theta
// below 1e-6 has not halved within 8 updates (the stop rule is applied on the
// device, lgf_reduce.cuh).  Without profiling the whole queue is one graph
// launch (a device-side while loop); with profiling, which needs events
// between launches, the host queues iterations and checks between batches of
// them.  Both run the same kernels and stop at the same update.  Returns
// LGF_OK / error and the number of updates through *done_iters.
int run_fix(lgf_handle h, Engine& e, double tol, int max_iter, bool stall_check,
            int* done_iters, bool* converged) {
  *converged = false;
  if (!h->profiling && kDeviceLoops) {
    lgf_ctx::DevLoop& l = h->loops[loop_kind(h, e)];
    if (!l.exec) {
      int rc = build_loop(h, e, l);
      if (rc) return rc;
    }
    int rc = reset_state(h, tol, max_iter, true, stall_check, true, l.cond);
    if (rc) return rc;
    LGF_CUDA(h, cudaGraphLaunch(l.exec, h->stream));
    rc = sync_state(h);
    if (rc) return rc;
    const DevState& s = *h->st_host;
    h->launches += (long long)(s.iters + 1) * l.launches;
    if (s.nonfinite) return fail(h, LGF_ERR_NONFINITE, "F or theta is not finite (non-SU(3) or NaN input links?)");
    *done_iters = s.iters;
    h->hist_n = s.iters + 1 < h->hist_cap ? s.iters + 1 : h->hist_cap;
    *converged = s.theta < tol;
    return LGF_OK;
  }
  int rc = reset_state(h, tol, max_iter, true, stall_check);
  if (rc) return rc;
  long long queued = 0;
  // queue length: 8 iterations first, then as many as the measured contraction
  // rate predicts are still needed (+1), at most LGF_CHECK_EVERY; iterations
  // queued past the stop decision cost only empty launches, but they do cost
  int k = h->check_every < 8 ? h->check_every : 8;
  double prev_theta = -1.0;
  int prev_iters = 0;
  for (;;) {
    const long long room = (long long)max_iter + 1 - queued;
    if (k > room) k = (int)room;
    if (k < 1) k = 1;
    for (int i = 0; i < k; ++i) {
      rc = queue_iteration(h, e);
      if (rc) return rc;
    }
    queued += k;
    rc = sync_state(h);
    if (rc) return rc;
    const DevState& s = *h->st_host;
    if (s.nonfinite) return fail(h, LGF_ERR_NONFINITE, "F or theta is not finite (non-SU(3) or NaN input links?)");
    if (s.done || queued >= (long long)max_iter + 1) break;
    // predict the iterations still needed from the last interval
    int next = h->check_every;
    const int dn = s.iters - prev_iters;
    if (prev_theta > 0.0 && dn > 0 && s.theta < prev_theta && s.theta > 0.0) {
      const double r = pow(s.theta / prev_theta, 1.0 / dn);
      if (r < 0.999) {
        const double need = log(tol / s.theta) / log(r);
        next = need < 1.0 ? 1 : (int)ceil(need) + 1;
      }
    }
    k = next < h->check_every ? next : h->check_every;
    prev_theta = s.theta;
    prev_iters = s.iters;
  }
  const DevState& s = *h->st_host;
  *done_iters = s.iters;
  h->hist_n = s.iters + 1 < h->hist_cap ? s.iters + 1 : h->hist_cap;
  *converged = s.theta < tol;
  return LGF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// autotuner: FFT pipeline per lattice shape and precision
// ---------------------------------------------------------------------------
namespace {


// Time every FFT schedule that applies to engine e -- each pipeline, and for
// the register plane pipeline each z-t tile width and radix order -- on the
// Fourier acceleration of its packed-gradient buffer (scratch between
// iterations), and return the fastest.  Results are kept per (precision,
// shape) for the process.
int tune_engine(lgf_handle h, Engine& e, int reps, TuneEntry* out) {
  const auto key = std::make_tuple(e.prec, h->L[0], h->L[1], h->L[2], h->L[3]);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *out = it->second;
      return LGF_OK;
    }
  }
  LGF_CUDA(h, cudaMemsetAsync(e.D, 0, (size_t)4 * h->V * e.cbytes(), h->stream));
  std::vector<TuneEntry> cands;
  cands.push_back({1, 0, 0});
  if (e.axis) cands.push_back({2, 0, 0});
  if (e.plane) {
    const int b0 = e.prec == 4 ? 4 : 2;
    for (int bx : {0, 2 * b0})
      for (int ro : {0, 1, 2})
        if (plane_zt_schedule_supported(e.prec, h->L[0], h->L[2], h->L[3], bx, ro)) cands.push_back({3, bx, ro});
  }
  cudaEvent_t a, b;
  LGF_CUDA(h, cudaEventCreate(&a));
  LGF_CUDA(h, cudaEventCreate(&b));
  const int saved = h->fft_pipeline;
  const int saved_bx = e.zt_bx, saved_ro = e.zt_ro;
  const bool saved_prof = h->profiling;
  h->profiling = false;
  TuneEntry best = cands[0];
  int rc = LGF_OK;
  for (size_t c = 0; c < cands.size(); ++c) {
    h->fft_pipeline = cands[c].pipeline;
    e.zt_bx = cands[c].zt_bx;
    e.zt_ro = cands[c].zt_ro;
    for (int i = 0; i < 2 && !rc; ++i) rc = queue_accelerate(h, e, nullptr);
    if (rc) break;
    cudaEventRecord(a, h->stream);
    for (int i = 0; i < reps && !rc; ++i) rc = queue_accelerate(h, e, nullptr);
    cudaEventRecord(b, h->stream);
    if (rc) break;
    if (cudaEventSynchronize(b) != cudaSuccess) {
      rc = fail(h, LGF_ERR_CUDA, "autotune: event synchronisation failed");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cands[c].ms = (double)ms / reps;
    if (c == 0 || cands[c].ms < best.ms) best = cands[c];
  }
  h->fft_pipeline = saved;
  e.zt_bx = saved_bx;
  e.zt_ro = saved_ro;
  h->profiling = saved_prof;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  *out = best;
  return LGF_OK;
}

// ---------------------------------------------------------------------------
// the schedule cache as a JSON file: one object per line inside a list,
//   {"prec": 4, "L": [32, 32, 32, 32], "pipeline": 3, "zt_bx": 4, "zt_ro": 0, "ms": 0.0531}
// (prec in bytes per real).  The reader takes these lines back (any order,
// other lines ignored) and rejects values no engine could run.
// ---------------------------------------------------------------------------
bool json_int(const char* line, const char* name, int* out) {
  char pat[32];
  snprintf(pat, sizeof pat, "\"%s\"", name);
  const char* p = strstr(line, pat);
  if (!p) return false;
  p = strchr(p + strlen(pat), ':');
  if (!p) return false;
  char* end = nullptr;
  const long v = strtol(p + 1, &end, 10);
  if (end == p + 1) return false;
  *out = (int)v;
  return true;
}

bool json_extents(const char* line, int L[4]) {
  const char* p = strstr(line, "\"L\"");
  if (!p) return false;
  p = strchr(p, '[');
  if (!p) return false;
  ++p;
  for (int a = 0; a < 4; ++a) {
    char* end = nullptr;
    const long v = strtol(p, &end, 10);
    if (end == p) return false;
    L[a] = (int)v;
    p = end;
    while (*p == ' ' || *p == ',') ++p;
  }
  return *p == ']';
}

bool valid_entry(int prec, const int L[4], const TuneEntry& t) {
  if (prec != 4 && prec != 8) return false;
  for (int a = 0; a < 4; ++a)
    if (L[a] < 2 || L[a] > kMaxL) return false;
  if (t.pipeline < 1 || t.pipeline > 3) return false;
  if (t.pipeline != 3) return t.zt_bx == 0 && t.zt_ro == 0;
  return plane_pipeline_supported(prec, L[0], L[1], L[2], L[3]) &&
         plane_zt_schedule_supported(prec, L[0], L[2], L[3], t.zt_bx, t.zt_ro);
}

int tune_load_file(const char* path, int* n_out) {
  FILE* f = fopen(path, "r");
  if (!f) return LGF_ERR_ARG;
  char line[512];
  int n = 0;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  while (fgets(line, sizeof line, f)) {
    int prec = 0, L[4];
    TuneEntry t;
    if (!json_int(line, "prec", &prec) || !json_extents(line, L) || !json_int(line, "pipeline", &t.pipeline) ||
        !json_int(line, "zt_bx", &t.zt_bx) || !json_int(line, "zt_ro", &t.zt_ro))
      continue;
    const char* m = strstr(line, "\"ms\"");
    if (m && (m = strchr(m, ':'))) t.ms = strtod(m + 1, nullptr);
    if (!valid_entry(prec, L, t)) continue;
    g_tune_cache[std::make_tuple(prec, L[0], L[1], L[2], L[3])] = t;
    ++n;
  }
  fclose(f);
  g_tune_apply_at_create = true;
  if (n_out) *n_out = n;
  return LGF_OK;
}

int tune_save_file(const char* path) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return LGF_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    fprintf(f, "{\"lgf_fft_schedules\": [\n");
    size_t i = 0;
    for (const auto& kv : g_tune_cache) {
      const TuneKey& k = kv.first;
      const TuneEntry& t = kv.second;
      fprintf(f, " {\"prec\": %d, \"L\": [%d, %d, %d, %d], \"pipeline\": %d, \"zt_bx\": %d, \"zt_ro\": %d, \"ms\": %.6f}%s\n",
              std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), t.pipeline, t.zt_bx,
              t.zt_ro, t.ms, ++i < g_tune_cache.size() ? "," : "");
    }
    fprintf(f, "]}\n");
  }
  const bool ok = fclose(f) == 0 && rename(tmp.c_str(), path) == 0;
  return ok ? LGF_OK : LGF_ERR_ARG;
}

}  // namespace

// ---------------------------------------------------------------------------
// batches: many lattices (of any sizes) iterated together from CUDA graphs
// ---------------------------------------------------------------------------
struct lgf_batch_ctx {
  std::vector<lgf_handle> h;
  std::vector<cudaStream_t> streams;  // capture streams of the lanes (at most one per member)
  cudaStream_t main = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;        // source of exec (holds the members' loop conditions)
  int lanes = 0;                      // parallel graph branches (0: one per member)
  std::vector<int> exec_members;      // members captured in exec
  std::vector<long long> exec_launches;  // kernels per member per graph launch
  std::string err;
};

namespace {

int bfail(lgf_batch b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

#define LGF_BCUDA(b, call)                                                                             \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return bfail((b), LGF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void drop_graph(lgf_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->exec_members.clear();
}

// One graph over the listed members: for each member a while node around one
// captured iteration of its current engine, stopped by the member's own
// on-device decision (lgf_reduce.cuh); the members' nodes run as parallel
// lanes (lgf_batch_set_lanes), the nodes of a lane one after another.  The
// loop conditions are returned in conds (one per member).
int capture(lgf_batch b, const std::vector<int>& members, std::vector<unsigned long long>& conds) {
  drop_graph(b);
  conds.assign(members.size(), 0);
  b->exec_launches.assign(members.size(), 0);
  const int nl = (b->lanes <= 0 || b->lanes > (int)members.size()) ? (int)members.size() : b->lanes;
  std::vector<size_t> order(members.size());
  for (size_t m = 0; m < order.size(); ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t a, size_t c) { return b->h[members[a]]->V > b->h[members[c]]->V; });
  std::vector<int64_t> load(nl, 0);
  std::vector<std::vector<size_t>> lane(nl);
  for (size_t m : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane[j].push_back(m);
    load[j] += b->h[members[m]]->V;
  }
  cudaGraph_t g = nullptr;
  LGF_BCUDA(b, cudaGraphCreate(&g, 0));
  int rc = LGF_OK;
  cudaError_t err = cudaSuccess;
  for (int j = 0; j < nl && !rc && err == cudaSuccess; ++j) {
    cudaGraphNode_t prev = nullptr;
    for (size_t m : lane[j]) {
      lgf_handle h = b->h[members[m]];
      cudaGraphConditionalHandle cond = 0;
      cudaGraphNodeParams p = {};
      cudaGraphNode_t node = nullptr;
      err = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
      if (err != cudaSuccess) break;
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = cond;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      err = cudaGraphAddNode(&node, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &p);
      if (err != cudaSuccess) break;
      cudaStream_t ls = b->streams[j];
      cudaStream_t saved = h->stream;
      const bool prof = h->profiling;
      h->stream = ls;
      h->profiling = false;
      const long long l0 = h->launches;
      err = cudaStreamBeginCaptureToGraph(ls, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
      if (err == cudaSuccess) {
        rc = queue_iteration(h, *h->cur);
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(ls, &out);
        if (!rc && e2 != cudaSuccess) err = e2;
      }
      b->exec_launches[m] = h->launches - l0;
      h->launches = l0;
      h->stream = saved;
      h->profiling = prof;
      if (rc) {
        b->err = h->err;
        break;
      }
      conds[m] = cond;
      prev = node;
    }
  }
  if (!rc && err == cudaSuccess) err = cudaGraphInstantiate(&b->exec, g, 0);
  if (rc || err != cudaSuccess) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaGraphDestroy(g);
    return rc ? rc : bfail(b, LGF_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(err));
  }
  b->graph = g;
  b->exec_members = members;
  return LGF_OK;
}

// Reset the members' stop state (with their loop conditions) on the main
// stream.
int reset_members(lgf_batch b, const std::vector<int>& members, const std::vector<double>& tol,
                  const std::vector<int>& max_iter, const std::vector<char>& stall,
                  const std::vector<unsigned long long>& conds) {
  for (size_t m = 0; m < members.size(); ++m) {
    lgf_handle h = b->h[members[m]];
    DevState s{};
    s.max_iter = max_iter[m];
    s.tol = tol[m];
    s.hist = h->hist;
    s.hist_cap = h->hist_cap;
    s.stall = stall[m] ? 1 : 0;
    s.use_cond = 1;
    s.cond = conds[m];
    *h->st_host = s;
    LGF_BCUDA(b, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, b->main));
  }
  LGF_BCUDA(b, cudaStreamSynchronize(b->main));
  return LGF_OK;
}

int read_members(lgf_batch b, const std::vector<int>& members) {
  for (int i : members) {
    lgf_handle h = b->h[i];
    LGF_BCUDA(b, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, b->main));
  }
  LGF_BCUDA(b, cudaStreamSynchronize(b->main));
  return LGF_OK;
}

// Run the listed members until each has stopped (theta < tol, its update
// budget, or -- with stall_check -- theta below 1e-6 no longer halving within
// 8 updates): one launch of the batch graph, every member looping on the
// device until its own stop decision.
int run_members(lgf_batch b, const std::vector<int>& members, const std::vector<double>& tol,
                const std::vector<int>& max_iter, const std::vector<char>& stall_check) {
  if (members.empty()) return LGF_OK;
  std::vector<unsigned long long> conds;
  int rc = capture(b, members, conds);
  if (rc) return rc;
  rc = reset_members(b, members, tol, max_iter, stall_check, conds);
  if (rc) return rc;
  LGF_BCUDA(b, cudaGraphLaunch(b->exec, b->main));
  rc = read_members(b, members);
  if (rc) return rc;
  for (size_t m = 0; m < members.size(); ++m) {
    lgf_handle h = b->h[members[m]];
    const DevState& s = *h->st_host;
    h->launches += (long long)(s.iters + 1) * b->exec_launches[m];
    if (s.nonfinite)
      return bfail(b, LGF_ERR_NONFINITE, "member " + std::to_string(members[m]) + ": F or theta is not finite");
    h->hist_n = s.iters + 1 < h->hist_cap ? s.iters + 1 : h->hist_cap;
  }
  return LGF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// learned warm start
// ---------------------------------------------------------------------------
struct lgf_net_ctx {
  int device = 0;
  float* p = nullptr;  // FP32 master parameters [W1 b1 W2 b2 W3 b3]
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;  // gradient in the same layout
  void* W1 = nullptr;
  void* W2 = nullptr;
  void* W3 = nullptr;  // bf16, last layer 16 wide
  void *Wt1 = nullptr, *Wt2 = nullptr, *Wt3 = nullptr;  // the same K-major ([tap][out][in]) for the forward
  int* tc_err = nullptr;  // [0] set by a tensor-core convolution whose bounded wait expired,
                          // [1] the poll budget of the convolutions' stage waits
  float* b1 = nullptr;
  float* b2 = nullptr;
  float* b3 = nullptr;
  float* gW3p = nullptr;  // padded last-layer gradient
  float* gb3p = nullptr;
  int64_t vmax = 0;
  void *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *y3 = nullptr, *gc = nullptr, *ga2 = nullptr, *ga1 = nullptr;
  float* c = nullptr;  // FP32 [V][16] outputs of the last layer
  void* G0 = nullptr;  // FP32 9 planes: g0 for the training signal
  long long step = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  std::string err;
};

namespace {

constexpr int kW1 = 81 * 48 * 32, kW2 = 81 * 32 * 32, kW3 = 81 * 32 * 8;
constexpr int kOB1 = kW1, kOW2 = kOB1 + 32, kOB2 = kOW2 + kW2, kOW3 = kOB2 + 32, kOB3 = kOW3 + kW3;

int nfail(lgf_net n, int code, const std::string& msg) {
  if (n) n->err = msg;
  else g_last_create_error = msg;
  return code;
}

#define LGF_NCUDA(n, call)                                                                                  \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess) return nfail((n), LGF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void* net_alloc(lgf_net n, size_t bytes) {
  void* q = nullptr;
  if (g_alloc.alloc) {
    q = g_alloc.alloc(bytes, n->device, nullptr, g_alloc.user);
  } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    q = nullptr;
  }
  if (q) n->allocs.push_back({q, bytes});
  return q;
}

void net_free(lgf_net n, void* q) {
  for (size_t i = 0; i < n->allocs.size(); ++i)
    if (n->allocs[i].first == q) {
      if (g_alloc.free_fn)
        g_alloc.free_fn(q, n->allocs[i].second, n->device, nullptr, g_alloc.user);
      else
        cudaFree(q);
      n->allocs.erase(n->allocs.begin() + i);
      return;
    }
}

// SplitMix64 (Steele, Lea & Flood 2014) of a counter, then Box-Muller
uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double normal_at(uint64_t seed, uint64_t i) {
  const uint64_t k = seed * 0x100000000ull + i;
  const double u1 = ((double)(splitmix64(2 * k) >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(splitmix64(2 * k + 1) >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

int net_pack(lgf_net n, cudaStream_t s) {
  LGF_NCUDA(n, warm::launch_pack_weights(n->p, n->W1, n->W2, n->W3, n->b1, n->b2, n->b3, n->Wt1, n->Wt2, n->Wt3, s));
  return LGF_OK;
}

int net_buffers(lgf_net n, int64_t V) {
  if (V <= n->vmax) return LGF_OK;
  for (void* q : {n->x0, n->a1, n->a2, n->y3, n->gc, n->ga2, n->ga1, (void*)n->c, n->G0})
    if (q) net_free(n, q);
  const size_t b = 2;  // bytes per bf16
  n->x0 = net_alloc(n, (size_t)V * 48 * b);
  n->a1 = net_alloc(n, (size_t)V * 32 * b);
  n->a2 = net_alloc(n, (size_t)V * 32 * b);
  n->y3 = net_alloc(n, (size_t)V * 16 * b);
  n->gc = net_alloc(n, (size_t)V * 16 * b);
  n->ga2 = net_alloc(n, (size_t)V * 32 * b);
  n->ga1 = net_alloc(n, (size_t)V * 32 * b);
  n->c = static_cast<float*>(net_alloc(n, (size_t)V * 16 * sizeof(float)));
  n->G0 = net_alloc(n, (size_t)V * 9 * 8);
  if (!n->x0 || !n->a1 || !n->a2 || !n->y3 || !n->gc || !n->ga2 || !n->ga1 || !n->c || !n->G0) {
    n->vmax = 0;
    return nfail(n, LGF_ERR_OOM, "device allocation of the network activations failed");
  }
  n->vmax = V;
  return LGF_OK;
}

int net_check_handle(lgf_net n, lgf_handle h) {
  if (!n || !h) return LGF_ERR_ARG;
  if (!h->mixed || !h->e32.grep || h->cur != &h->e32)
    return nfail(n, LGF_ERR_ARG, "the warm start needs an FP32 handle in gauge representation before its FP64 tail");
  if (!h->loaded) return nfail(n, LGF_ERR_ARG, "no links loaded");
  if (h->V % 16 != 0) return nfail(n, LGF_ERR_ARG, "the lattice volume must be a multiple of 16");
  return net_buffers(n, h->V);
}

int net_forward(lgf_net n, lgf_handle h) {
  cudaStream_t s = h->stream;
  LGF_NCUDA(n, warm::launch_features(h->e32.nc, h->e32.U, n->x0, h->geo, s));
  LGF_NCUDA(n, warm::launch_conv_fwd_tc(1, n->x0, n->Wt1, n->b1, n->a1, nullptr, h->geo, n->tc_err, s));
  LGF_NCUDA(n, warm::launch_conv_fwd_tc(2, n->a1, n->Wt2, n->b2, n->a2, nullptr, h->geo, n->tc_err, s));
  LGF_NCUDA(n, warm::launch_conv_fwd_tc(3, n->a2, n->Wt3, n->b3, n->y3, n->c, h->geo, n->tc_err, s));
  h->launches += 4;
  return LGF_OK;
}

// after the stream has been synchronised: LGF_ERR_TIMEOUT (and the flag
// cleared) if a tensor-core convolution gave up a bounded wait
int net_check_tc(lgf_net n) {
  int flag = 0;
  LGF_NCUDA(n, cudaMemcpy(&flag, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag == 0) return LGF_OK;
  LGF_NCUDA(n, cudaMemset(n->tc_err, 0, sizeof(int)));
  return nfail(n, LGF_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
}

}  // namespace

extern "C" {

int lgf_set_allocator(lgf_alloc_fn alloc, lgf_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return LGF_ERR_ARG;
  g_alloc.alloc = alloc;
  g_alloc.free_fn = free_fn;
  g_alloc.user = user;
  return LGF_OK;
}

int lgf_create(int Lx, int Ly, int Lz, int Lt, int dtype, lgf_handle* out) {
  if (!out) return fail(nullptr, LGF_ERR_ARG, "out is NULL");
  *out = nullptr;
  const int Ls[4] = {Lx, Ly, Lz, Lt};
  if (dtype < LGF_F64 || dtype > LGF_F64_R12) return fail(nullptr, LGF_ERR_ARG, "unknown dtype");
  FftGeom fg{};
  for (int a = 0; a < 4; ++a) {
    if (!make_axis_plan(Ls[a], &fg.ax[a]))
      return fail(nullptr, LGF_ERR_ARG,
                  "each lattice extent must be in [2, 64] and a product of 2, 3 and 5; got " +
                      std::to_string(Ls[a]));
    fg.L[a] = Ls[a];
  }
  lgf_ctx* h = new (std::nothrow) lgf_ctx();
  if (!h) return fail(nullptr, LGF_ERR_OOM, "host allocation failed");
  h->dtype = dtype;
  h->mixed = (dtype == LGF_F32 || dtype == LGF_F32_R12);
  int64_t V = 1;
  for (int a = 0; a < 4; ++a) {
    h->L[a] = Ls[a];
    h->geo.L[a] = Ls[a];
    h->geo.stride[a] = V;
    V *= Ls[a];
  }
  h->V = V;
  h->geo.V = V;
  geom_init_rcp(h->geo);
  fg.V = V;
  double p2max = 0.0;
  for (int a = 0; a < 4; ++a) {
    double m = 0.0;
    for (int k = 0; k < Ls[a]; ++k) {
      const double sk = sin(M_PI * (double)k / (double)Ls[a]);
      m = fmax(m, 4.0 * sk * sk);
    }
    p2max += m;
  }
  fg.p2max = p2max;
  auto bail = [&](int code) {
    std::string msg = h->err;
    dev_free_all(h);
    if (h->st_host) cudaFreeHost(h->st_host);
    delete h;
    g_last_create_error = msg;
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    h->err = "no CUDA device";
    return bail(LGF_ERR_CUDA);
  }
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);

  // engines: FP64 always (working engine of FP64 handles, tail of mixed ones)
  h->e64.prec = 8;
  h->e64.nc = (dtype == LGF_F64_R12) ? 6 : 9;
  if (h->mixed) {
    h->e64.nc = 9;
    h->e32.prec = 4;
    h->e32.nc = (dtype == LGF_F32_R12) ? 6 : 9;
  }
  // FFT tiling: Bx consecutive x (>= 32 bytes of complex data when Lx allows)
  auto pick = [&](Engine& e) -> bool {
    FftGeom g = fg;
    const int want = e.prec == 8 ? 2 : 4;
    int bx = 1;
    for (int b = want; b >= 1; b >>= 1)
      if (Lx % b == 0) {
        bx = b;
        break;
      }
    g.Bx = bx;
    g.Pxy = Lx + 1;
    g.Pt = bx * (Lz + 1);
    e.fg = g;
    return fft_xy_smem(g, e.prec) <= (size_t)smem_optin && fft_zt_smem(g, e.prec) <= (size_t)smem_optin;
  };
  if (!pick(h->e64) || (h->mixed && !pick(h->e32))) {
    h->err = "lattice planes too large for the shared-memory FFT";
    return bail(LGF_ERR_ARG);
  }
  // the opt-in limit is process-wide per kernel: always raise it to the device maximum
  cudaError_t e = fft_set_smem_limits(8, smem_optin, smem_optin);
  if (e == cudaSuccess) e = fft_set_smem_limits(4, smem_optin, smem_optin);
  if (e == cudaSuccess) e = axis_pass_init();
  if (e == cudaSuccess) e = plane_pipeline_init();
  if (e != cudaSuccess) {
    cuda_fail(h, e, "cudaFuncSetAttribute");
    return bail(LGF_ERR_CUDA);
  }

  int rc = alloc_engine(h, h->e64);
  if (!rc && h->mixed) rc = alloc_engine(h, h->e32);
  if (!rc) {
    apply_cached_schedule(h, h->e64);
    if (h->mixed) apply_cached_schedule(h, h->e32);
  }
  if (rc) return bail(rc);
  h->cur = h->mixed ? &h->e32 : &h->e64;
  if (h->mixed) {
    h->G = dev_alloc(h, (size_t)h->e32.nc * V * h->e32.cbytes());
    h->Uorig = static_cast<double*>(dev_alloc(h, (size_t)4 * 9 * V * 16));
    if (!h->G || !h->Uorig) {
      h->err = "device allocation failed";
      return bail(LGF_ERR_OOM);
    }
  }
  h->nblk = gradient_blocks(V);
  h->partial = static_cast<double2*>(dev_alloc(h, (size_t)partial_capacity(V) * sizeof(double2)));
  h->st = static_cast<DevState*>(dev_alloc(h, sizeof(DevState)));
  h->sin2 = static_cast<double*>(dev_alloc(h, 4 * kMaxL * sizeof(double)));
  h->hist_cap = 1 << 16;
  h->hist = static_cast<double*>(dev_alloc(h, (size_t)h->hist_cap * sizeof(double)));
  if (!h->partial || !h->st || !h->sin2 || !h->hist) {
    h->err = "device allocation failed";
    return bail(LGF_ERR_OOM);
  }
  if (cudaMallocHost(&h->st_host, sizeof(DevState)) != cudaSuccess) {
    h->st_host = nullptr;
    h->err = "pinned host allocation failed";
    return bail(LGF_ERR_OOM);
  }
  std::vector<double> s2(4 * kMaxL, 0.0);
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < Ls[a]; ++k) {
      const long double sk = sinl(3.14159265358979323846264338327950288L * (long double)k / (long double)Ls[a]);
      s2[a * kMaxL + k] = (double)(4.0L * sk * sk);
    }
  if (cudaMemcpy(h->sin2, s2.data(), s2.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    h->err = "copy of the momentum table failed";
    return bail(LGF_ERR_CUDA);
  }
  if (reset_state(h, -1.0, 0, false) || cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->err = "state initialisation failed";
    return bail(LGF_ERR_CUDA);
  }
  *out = h;
  return LGF_OK;
}

int lgf_destroy(lgf_handle h) {
  if (!h) return LGF_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  drop_loops(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
  dev_free_all(h);
  if (h->st_host) cudaFreeHost(h->st_host);
  delete h;
  return LGF_OK;
}

int lgf_set_stream(lgf_handle h, void* cuda_stream) {
  if (!h) return LGF_ERR_ARG;
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return LGF_OK;
}

int lgf_set_param(lgf_handle h, int key, double value) {
  if (!h) return LGF_ERR_ARG;
  drop_loops(h);  // captured loop bodies hold the parameters
  switch (key) {
    case LGF_ALPHA:
      if (!(value > 0.0 && value <= 0.125)) return fail(h, LGF_ERR_ARG, "alpha must lie in (0, 0.125]");
      h->alpha = value;
      return LGF_OK;
    case LGF_CHECK_EVERY:
      if (!(value >= 1 && value <= 4096)) return fail(h, LGF_ERR_ARG, "check_every must lie in [1, 4096]");
      h->check_every = (int)value;
      return LGF_OK;
    case LGF_TAIL_THETA:
      if (!(value > 0.0)) return fail(h, LGF_ERR_ARG, "tail theta must be positive");
      h->tail_theta = value;
      return LGF_OK;
    case LGF_TAIL_MAX_FP32:
      h->tail_max32 = (long long)value;
      return LGF_OK;
    case LGF_REUNIT_FP64:
      h->reunit_fp64 = value != 0.0;
      return LGF_OK;
    case LGF_FFT_PIPELINE:
      if (!(value >= 0 && value <= 3)) return fail(h, LGF_ERR_ARG, "FFT pipeline must be 0, 1, 2 or 3");
      h->fft_pipeline = (int)value;
      return LGF_OK;
    case LGF_LINK_UPDATE:
      h->explicit_fp32 = value != 0.0;
      return LGF_OK;
    case LGF_TRACK_G:
      h->track_g = value != 0.0;
      return LGF_OK;
    case LGF_EXP_ORDER:
      if (!(value == 0.0 || value == 1.0)) return fail(h, LGF_ERR_ARG, "exp order must be 0 or 1");
      h->exp_order = (int)value;
      return LGF_OK;
    case LGF_TAIL_MODE:
      if (!(value == 0.0 || value == 1.0 || value == 2.0)) return fail(h, LGF_ERR_ARG, "tail mode must be 0, 1 or 2");
      h->tail_mode = (int)value;
      return LGF_OK;
    default:
      return fail(h, LGF_ERR_ARG, "unknown parameter key");
  }
}

// Queue the re-layout of device AoS links into the handle's storage on its
// stream (no host synchronisation); the handle counts as loaded from here on.
static int queue_load(lgf_handle h, const double* aos) {
  const int64_t V = h->V;
  // the FP32 engine's update mode is fixed at the load; loop bodies captured
  // for the other mode are dropped
  if (h->mixed && h->e32.grep != !h->explicit_fp32) drop_loops(h);
  const bool staged = ((uintptr_t)aos & 15) == 0;  // 16-byte copies of the input chunks
  if (h->mixed) {
    if (staged) {  // one read of the input for both copies
      LGF_LAUNCH(h, LGF_K_OTHER, launch_load_aos(9, h->e32.nc, aos, h->Uorig, h->e32.U, V, h->stream));
    } else {
      LGF_LAUNCH(h, LGF_K_OTHER, launch_aos_to_soa(8, 9, aos, h->Uorig, V, 4, h->stream));
      LGF_LAUNCH(h, LGF_K_OTHER, launch_aos_to_soa(4, h->e32.nc, aos, h->e32.U, V, 4, h->stream));
    }
    LGF_LAUNCH(h, LGF_K_OTHER, launch_set_identity(4, h->e32.nc, h->G, V, h->stream));
    h->e32.grep = !h->explicit_fp32;
    h->defect = false;
    h->df = false;
    h->cur = &h->e32;
  } else if (staged) {
    LGF_LAUNCH(h, LGF_K_OTHER, launch_load_aos(h->e64.nc, 0, aos, h->e64.U, nullptr, V, h->stream));
  } else {
    LGF_LAUNCH(h, LGF_K_OTHER, launch_aos_to_soa(8, h->e64.nc, aos, h->e64.U, V, 4, h->stream));
  }
  if (!h->mixed) {
    // LGF_TRACK_G takes effect here; a change of it drops the captured loops
    if (h->g64_track != h->track_g) drop_loops(h);
    h->g64_track = false;
    if (h->track_g) {
      if (!h->G) h->G = dev_alloc(h, (size_t)h->e64.nc * V * 16);
      if (!h->G) return fail(h, LGF_ERR_OOM, "device allocation of the tracked gauge transformation failed");
      LGF_LAUNCH(h, LGF_K_OTHER, launch_set_identity(8, h->e64.nc, h->G, V, h->stream));
      h->g64_track = true;
    }
  }
  h->g_valid = h->mixed || h->g64_track;
  h->loaded = true;
  h->total_updates = 0;
  return LGF_OK;
}

static int load_from_device_aos(lgf_handle h, const double* aos) {
  int rc = queue_load(h, aos);
  if (rc) return rc;
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

// Device address of host memory the GPU reads and writes directly (pinned,
// registered with CUDA, 16-byte aligned), or null: the link load and store
// then move the host array once, inside their layout kernels, instead of a
// staging copy plus a device-side conversion.
static double* host_direct(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || ((uintptr_t)a.devicePointer & 15) != 0) return nullptr;
  return static_cast<double*>(a.devicePointer);
}

int lgf_load_links(lgf_handle h, const double* host_aos) {
  if (!h || !host_aos) return LGF_ERR_ARG;
  if (const double* direct = host_direct(host_aos)) return load_from_device_aos(h, direct);
  int rc = ensure_staging(h);
  if (rc) return rc;
  LGF_CUDA(h, cudaMemcpyAsync(h->staging, host_aos, (size_t)h->V * 72 * sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
  return load_from_device_aos(h, h->staging);
}

int lgf_load_links_device(lgf_handle h, const double* dev_aos) {
  if (!h || !dev_aos) return LGF_ERR_ARG;
  return load_from_device_aos(h, dev_aos);
}

// Queue the current links, as FP64 AoS, into dst (device memory, or host
// memory the device writes directly) on the handle's stream.
static int queue_store(lgf_handle h, double* dst) {
  Engine& e = *h->cur;
  if (&e == &h->e64 && h->df)
    LGF_LAUNCH(h, LGF_K_OTHER, launch_store_aos_df(h->Udf, h->eta, h->geo, dst, h->stream));
  else if (e.grep)
    LGF_LAUNCH(h, LGF_K_OTHER, launch_materialize(e.nc, e.U, h->G, dst, h->geo, h->stream));
  else
    LGF_LAUNCH(h, LGF_K_OTHER, launch_store_aos(e.prec, e.nc, e.U, dst, h->V, h->stream));
  return LGF_OK;
}

int lgf_store_links(lgf_handle h, double* host_aos) {
  if (!h || !host_aos) return LGF_ERR_ARG;
  if (!h->loaded) return fail(h, LGF_ERR_ARG, "no links loaded");
  double* direct = host_direct(host_aos);
  if (!direct) {
    int rc = ensure_staging(h);
    if (rc) return rc;
  }
  int rc = queue_store(h, direct ? direct : h->staging);
  if (rc) return rc;
  if (!direct)
    LGF_CUDA(h, cudaMemcpyAsync(host_aos, h->staging, (size_t)h->V * 72 * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

int lgf_store_gauge(lgf_handle h, double* host_g) {
  if (!h || !host_g) return LGF_ERR_ARG;
  if (!h->loaded) return fail(h, LGF_ERR_ARG, "no links loaded");
  if (!h->g_valid)
    return fail(h, LGF_ERR_ARG,
                "the gauge transformation is not tracked (FP64 handles: set LGF_TRACK_G before the load; mixed "
                "handles lose it in the FP64-link tails and after lgf_probe on the double-float tail)");
  double* direct = host_direct(host_g);
  if (!direct) {
    int rc = ensure_staging(h);
    if (rc) return rc;
  }
  double* dst = direct ? direct : h->staging;
  if (h->mixed && h->cur == &h->e64 && h->df)
    LGF_LAUNCH(h, LGF_K_OTHER, launch_store_gauge_df(h->e64.g, h->eta, h->V, dst, h->stream));
  else if (h->mixed)
    LGF_LAUNCH(h, LGF_K_OTHER, launch_soa_to_aos(4, h->e32.nc, h->G, dst, h->V, 1, h->stream));
  else
    LGF_LAUNCH(h, LGF_K_OTHER, launch_soa_to_aos(8, h->e64.nc, h->G, dst, h->V, 1, h->stream));
  if (!direct)
    LGF_CUDA(h, cudaMemcpyAsync(host_g, h->staging, (size_t)h->V * 18 * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

int lgf_iterate(lgf_handle h, int n) {
  if (!h || n < 0) return LGF_ERR_ARG;
  if (!h->loaded) return fail(h, LGF_ERR_ARG, "no links loaded");
  int rc = reset_state(h, -1.0, n, false);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    rc = queue_iteration(h, *h->cur);
    if (rc) return rc;
  }
  rc = sync_state(h);
  if (rc) return rc;
  if (h->st_host->nonfinite) return fail(h, LGF_ERR_NONFINITE, "F or theta is not finite");
  h->total_updates += h->st_host->iters;
  return LGF_OK;
}

int lgf_fix(lgf_handle h, double theta_tol, int max_iter, int* iters_out) {
  if (!h || max_iter < 0 || !(theta_tol > 0.0)) return LGF_ERR_ARG;
  if (!h->loaded) return fail(h, LGF_ERR_ARG, "no links loaded");
  if (iters_out) *iters_out = 0;
  h->last_n32 = h->last_n64 = 0;
  int n1 = 0, n2 = 0;
  bool conv = false;
  int rc;
  if (h->mixed && h->cur == &h->e32) {
    // FP32 phase; G has been accumulated since the load
    const double tol32 = theta_tol > h->tail_theta ? theta_tol : h->tail_theta;
    int cap32 = max_iter;
    if (h->tail_max32 >= 0 && h->tail_max32 < cap32) cap32 = (int)h->tail_max32;
    rc = run_fix(h, h->e32, tol32, cap32, true, &n1, &conv);
    if (rc) return rc;
    h->total_updates += n1;
    h->last_n32 = n1;
    if (conv && h->st_host->theta < theta_tol) {
      if (iters_out) *iters_out = n1;
      return LGF_OK;
    }
    rc = queue_tail_start(h);
    if (rc) return rc;
  }
  const int left = max_iter - n1;
  rc = run_fix(h, *h->cur, theta_tol, left, false, &n2, &conv);
  if (rc) return rc;
  h->total_updates += n2;
  if (h->cur == &h->e64)
    h->last_n64 = n2;
  else
    h->last_n32 += n2;
  if (iters_out) *iters_out = n1 + n2;
  return conv ? LGF_OK : fail(h, LGF_ERR_NOT_CONVERGED, "max_iter reached with theta >= tol");
}

// ---------------------------------------------------------------------------
// streamed fixing of an ensemble (lgf_fix_stream)
// ---------------------------------------------------------------------------
namespace {

// Streams and events of one lgf_fix_stream call, released on every return
// path after all the work queued on them has finished.
struct StreamCtx {
  cudaStream_t cin = nullptr, cout = nullptr;  // host -> device and device -> host copies
  cudaEvent_t in_done[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
  lgf_handle H[2] = {nullptr, nullptr};
  ~StreamCtx() {
    if (cin) cudaStreamSynchronize(cin);
    if (cout) cudaStreamSynchronize(cout);
    for (lgf_handle h : H)
      if (h) cudaStreamSynchronize(h->stream);
    for (int s = 0; s < 2; ++s)
      for (cudaEvent_t ev : {in_done[s], in_free[s], out_ready[s], out_free[s]})
        if (ev) cudaEventDestroy(ev);
    if (cin) cudaStreamDestroy(cin);
    if (cout) cudaStreamDestroy(cout);
  }
  bool create() {
    if (cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (int s = 0; s < 2; ++s)
      for (cudaEvent_t* ev : {&in_done[s], &in_free[s], &out_ready[s], &out_free[s]})
        if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
  }
};

int ensure_staging_out(lgf_handle h) {
  if (h->staging_out) return LGF_OK;
  h->staging_out = static_cast<double*>(dev_alloc(h, (size_t)h->V * 72 * sizeof(double)));
  if (!h->staging_out) return fail(h, LGF_ERR_OOM, "device allocation of the result staging buffer failed");
  return LGF_OK;
}

}  // namespace

int lgf_fix_stream(lgf_handle h0, lgf_handle h1, int n, const double* const* host_in, double* const* host_out,
                   double theta_tol, int max_iter, int* iters_out) {
  if (!h0) return LGF_ERR_ARG;
  if (!h1 || h1 == h0) return fail(h0, LGF_ERR_ARG, "lgf_fix_stream: needs two distinct handles");
  if (n < 0 || max_iter < 0 || !(theta_tol > 0.0)) return fail(h0, LGF_ERR_ARG, "lgf_fix_stream: bad n, tol or max_iter");
  if (n > 0 && (!host_in || !host_out)) return fail(h0, LGF_ERR_ARG, "lgf_fix_stream: null configuration array");
  for (int a = 0; a < 4; ++a)
    if (h0->L[a] != h1->L[a]) return fail(h0, LGF_ERR_ARG, "lgf_fix_stream: the handles' lattices differ");
  if (h0->dtype != h1->dtype || h0->device != h1->device)
    return fail(h0, LGF_ERR_ARG, "lgf_fix_stream: the handles' dtype or device differ");
  for (int k = 0; k < n; ++k)
    if (!host_in[k] || !host_out[k]) return fail(h0, LGF_ERR_ARG, "lgf_fix_stream: null configuration pointer");
  if (n == 0) return LGF_OK;
  const size_t bytes = (size_t)h0->V * 72 * sizeof(double);
  StreamCtx c;
  c.H[0] = h0;
  c.H[1] = h1;
  for (lgf_handle h : c.H) {
    int rc = ensure_staging(h);
    if (!rc) rc = ensure_staging_out(h);
    if (rc) return fail(h0, rc, h->err);
  }
  if (!c.create()) return fail(h0, LGF_ERR_CUDA, "lgf_fix_stream: stream or event creation failed");
  // Configuration k goes to handle k % 2.  Its input lands in that handle's
  // staging buffer once the re-layout of configuration k - 2 has read it, and
  // its re-layout is queued on that handle's stream before configuration
  // k - 1 starts fixing on the other handle, so that it runs alongside that
  // fix (after the store of configuration k - 2 in stream order).
  auto queue_in = [&](int k) -> int {
    const int s = k & 1;
    lgf_handle h = c.H[s];
    if (k >= 2) LGF_CUDA(h0, cudaStreamWaitEvent(c.cin, c.in_free[s], 0));
    LGF_CUDA(h0, cudaMemcpyAsync(h->staging, host_in[k], bytes, cudaMemcpyHostToDevice, c.cin));
    LGF_CUDA(h0, cudaEventRecord(c.in_done[s], c.cin));
    return LGF_OK;
  };
  lgf_handle where = h0;  // the handle whose call failed (its message is reported through h0)
  auto load_next = [&](int k) -> int {
    const int s = k & 1;
    lgf_handle h = c.H[s];
    LGF_CUDA(h0, cudaStreamWaitEvent(h->stream, c.in_done[s], 0));
    where = h;
    int r = queue_load(h, h->staging);
    if (r) return r;
    where = h0;
    LGF_CUDA(h0, cudaEventRecord(c.in_free[s], h->stream));
    return k + 2 < n ? queue_in(k + 2) : LGF_OK;
  };
  int rc = queue_in(0);
  if (!rc && n > 1) rc = queue_in(1);
  if (!rc) rc = load_next(0);
  if (rc) return where == h0 ? rc : fail(h0, rc, "lgf_fix_stream: " + where->err);
  bool all_converged = true;
  for (int k = 0; k < n && !rc; ++k) {
    const int s = k & 1;
    lgf_handle h = c.H[s];
    if (k + 1 < n && (rc = load_next(k + 1)) != LGF_OK) break;
    where = h;
    int it = 0;
    rc = lgf_fix(h, theta_tol, max_iter, &it);
    if (iters_out) iters_out[k] = it;
    if (rc == LGF_ERR_NOT_CONVERGED) {
      all_converged = false;
      rc = LGF_OK;
    }
    if (rc) break;
    // the result buffer of this handle is free once configuration k - 2 is out
    if (k >= 2) LGF_CUDA(h0, cudaStreamWaitEvent(h->stream, c.out_free[s], 0));
    if ((rc = queue_store(h, h->staging_out)) != LGF_OK) break;
    where = h0;
    LGF_CUDA(h0, cudaEventRecord(c.out_ready[s], h->stream));
    LGF_CUDA(h0, cudaStreamWaitEvent(c.cout, c.out_ready[s], 0));
    LGF_CUDA(h0, cudaMemcpyAsync(host_out[k], h->staging_out, bytes, cudaMemcpyDeviceToHost, c.cout));
    LGF_CUDA(h0, cudaEventRecord(c.out_free[s], c.cout));
  }
  if (rc) return where == h0 ? rc : fail(h0, rc, "lgf_fix_stream: " + where->err);
  LGF_CUDA(h0, cudaStreamSynchronize(c.cout));
  LGF_CUDA(h0, cudaStreamSynchronize(c.cin));
  return all_converged ? LGF_OK : fail(h0, LGF_ERR_NOT_CONVERGED, "lgf_fix_stream: max_iter reached with theta >= tol");
}

int lgf_functional(lgf_handle h, double* F, double* theta) {
  if (!h) return LGF_ERR_ARG;
  if (!h->loaded) return fail(h, LGF_ERR_ARG, "no links loaded");
  Engine& e = *h->cur;
  int rc = queue_gradient(h, e, 0);
  if (!rc) rc = sync_state(h);
  if (rc) return rc;
  if (F) *F = h->st_host->F;
  if (theta) *theta = h->st_host->theta;
  if (h->st_host->nonfinite) return fail(h, LGF_ERR_NONFINITE, "F or theta is not finite");
  return LGF_OK;
}

int lgf_probe(lgf_handle h, double* delta_packed, double* delta_tilde_packed, double* g) {
  if (!h) return LGF_ERR_ARG;
  if (!h->loaded) return fail(h, LGF_ERR_ARG, "no links loaded");
  int rc = materialize_df(h);
  if (rc) return rc;
  rc = ensure_staging(h);
  if (rc) return rc;
  Engine& e = *h->cur;
  const int64_t V = h->V;
  cudaStream_t s = h->stream;
  rc = queue_gradient(h, e, 0);
  if (rc) return rc;
  if (delta_packed) {
    LGF_LAUNCH(h, LGF_K_OTHER, launch_unpack_fields(e.prec, e.D, h->staging, V, s));
    LGF_CUDA(h, cudaMemcpyAsync(delta_packed, h->staging, (size_t)V * 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LGF_CUDA(h, cudaStreamSynchronize(s));
  }
  rc = queue_accelerate(h, e, nullptr);
  if (rc) return rc;
  if (e.grep)  // g only: G is left alone
    LGF_LAUNCH(h, LGF_K_BUILD_G, launch_gstep(e.nc, e.D, nullptr, e.g, V, 0.5 * h->alpha, h->reunit_fp64,
                                              h->exp_order == 0, nullptr, s));
  else
    LGF_LAUNCH(h, LGF_K_BUILD_G,
               launch_build_g(e.prec, e.nc, e.D, e.g, V, 0.5 * h->alpha, h->reunit_fp64, h->exp_order == 0, nullptr,
                              s));
  if (delta_tilde_packed) {
    LGF_LAUNCH(h, LGF_K_OTHER, launch_unpack_fields(e.prec, e.D, h->staging, V, s));
    LGF_CUDA(h, cudaMemcpyAsync(delta_tilde_packed, h->staging, (size_t)V * 8 * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    LGF_CUDA(h, cudaStreamSynchronize(s));
  }
  if (g) {
    LGF_LAUNCH(h, LGF_K_OTHER, launch_soa_to_aos(e.prec, e.nc, e.g, h->staging, V, 1, s));
    LGF_CUDA(h, cudaMemcpyAsync(g, h->staging, (size_t)V * 18 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  LGF_CUDA(h, cudaStreamSynchronize(s));
  return LGF_OK;
}

int lgf_fix_split(lgf_handle h, int* fp32_iters, int* fp64_iters) {
  if (!h) return LGF_ERR_ARG;
  if (fp32_iters) *fp32_iters = h->last_n32;
  if (fp64_iters) *fp64_iters = h->last_n64;
  return LGF_OK;
}

int lgf_autotune(lgf_handle h, int reps, int* chosen) {
  if (!h || reps < 1) return LGF_ERR_ARG;
  drop_loops(h);
  TuneEntry t64, t32;
  int rc = tune_engine(h, h->e64, reps, &t64);
  if (rc) return rc;
  h->e64.tuned = t64.pipeline;
  h->e64.zt_bx = t64.zt_bx;
  h->e64.zt_ro = t64.zt_ro;
  if (h->mixed) {
    rc = tune_engine(h, h->e32, reps, &t32);
    if (rc) return rc;
    h->e32.tuned = t32.pipeline;
    h->e32.zt_bx = t32.zt_bx;
    h->e32.zt_ro = t32.zt_ro;
  }
  if (chosen) *chosen = h->mixed ? t32.pipeline : t64.pipeline;
  const char* path = getenv("LGF_TUNE_CACHE");
  if (path && *path && tune_save_file(path) != LGF_OK)
    return fail(h, LGF_ERR_ARG, std::string("lgf_autotune: cannot write the tuning cache ") + path);
  return LGF_OK;
}

int lgf_tune_schedule(lgf_handle h, int engine, int* pipeline, int* zt_bx, int* zt_ro) {
  if (!h || (engine != 0 && engine != 1)) return LGF_ERR_ARG;
  if (engine == 1 && !h->mixed) return fail(h, LGF_ERR_ARG, "lgf_tune_schedule: the handle has no FP32 engine");
  const Engine& e = engine == 1 ? h->e32 : h->e64;
  if (pipeline) *pipeline = pick_pipeline(h, e);
  if (zt_bx) *zt_bx = e.zt_bx;
  if (zt_ro) *zt_ro = e.zt_ro;
  return LGF_OK;
}

int lgf_set_schedule(lgf_handle h, int engine, int pipeline, int zt_bx, int zt_ro) {
  if (!h || (engine != 0 && engine != 1)) return LGF_ERR_ARG;
  if (engine == 1 && !h->mixed) return fail(h, LGF_ERR_ARG, "lgf_set_schedule: the handle has no FP32 engine");
  Engine& e = engine == 1 ? h->e32 : h->e64;
  TuneEntry t;
  t.pipeline = pipeline;
  t.zt_bx = zt_bx;
  t.zt_ro = zt_ro;
  if (!valid_entry(e.prec, h->L, t) || (pipeline == 2 && !e.axis))
    return fail(h, LGF_ERR_ARG, "lgf_set_schedule: schedule does not apply to this lattice and precision");
  drop_loops(h);
  e.tuned = pipeline;
  e.zt_bx = zt_bx;
  e.zt_ro = zt_ro;
  return LGF_OK;
}

int lgf_tune_load(const char* path, int* n_loaded) {
  if (!path) return LGF_ERR_ARG;
  const int rc = tune_load_file(path, n_loaded);
  if (rc) set_global_error(std::string("lgf_tune_load: cannot read ") + path);
  return rc;
}

int lgf_tune_save(const char* path) {
  if (!path) return LGF_ERR_ARG;
  const int rc = tune_save_file(path);
  if (rc) set_global_error(std::string("lgf_tune_save: cannot write ") + path);
  return rc;
}

int lgf_tune_lookup(int prec_bytes, int Lx, int Ly, int Lz, int Lt, int* pipeline, int* zt_bx, int* zt_ro) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune_cache.find(std::make_tuple(prec_bytes, Lx, Ly, Lz, Lt));
  if (it == g_tune_cache.end()) return LGF_ERR_ARG;
  if (pipeline) *pipeline = it->second.pipeline;
  if (zt_bx) *zt_bx = it->second.zt_bx;
  if (zt_ro) *zt_ro = it->second.zt_ro;
  return LGF_OK;
}

int lgf_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache.clear();
  g_tune_apply_at_create = false;
  return LGF_OK;
}

int lgf_batch_create(const lgf_handle* handles, int n, lgf_batch* out) {
  if (!out) return LGF_ERR_ARG;
  *out = nullptr;
  if (!handles || n < 1) return fail(nullptr, LGF_ERR_ARG, "lgf_batch_create: need at least one handle");
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return fail(nullptr, LGF_ERR_ARG, "lgf_batch_create: NULL handle");
    if (handles[i]->device != handles[0]->device)
      return fail(nullptr, LGF_ERR_ARG, "lgf_batch_create: all handles must live on one device");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(nullptr, LGF_ERR_ARG, "lgf_batch_create: a handle appears twice");
  }
  lgf_batch_ctx* b = new (std::nothrow) lgf_batch_ctx();
  if (!b) return fail(nullptr, LGF_ERR_OOM, "host allocation failed");
  b->h.assign(handles, handles + n);
  bool ok = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess;
  b->streams.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i) ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    lgf_batch_destroy(b);
    return fail(nullptr, LGF_ERR_CUDA, "lgf_batch_create: stream creation failed");
  }
  *out = b;
  return LGF_OK;
}

int lgf_batch_destroy(lgf_batch b) {
  if (!b) return LGF_ERR_ARG;
  if (b->main) cudaStreamSynchronize(b->main);
  drop_graph(b);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->main) cudaStreamDestroy(b->main);
  delete b;
  return LGF_OK;
}

int lgf_batch_iterate(lgf_batch b, int n) {
  if (!b || n < 0) return LGF_ERR_ARG;
  std::vector<int> all;
  for (int i = 0; i < (int)b->h.size(); ++i) {
    if (!b->h[i]->loaded) return bfail(b, LGF_ERR_ARG, "member " + std::to_string(i) + " has no links loaded");
    cudaStreamSynchronize(b->h[i]->stream);
    all.push_back(i);
  }
  std::vector<double> tol(all.size(), -1.0);
  std::vector<int> cap(all.size(), n);
  std::vector<char> stall(all.size(), 0);
  int rc = run_members(b, all, tol, cap, stall);
  if (rc) return rc;
  for (int i : all) b->h[i]->total_updates += b->h[i]->st_host->iters;
  return LGF_OK;
}

int lgf_batch_fix(lgf_batch b, double theta_tol, int max_iter, int* iters_out, int* converged_out) {
  if (!b || max_iter < 0 || !(theta_tol > 0.0)) return LGF_ERR_ARG;
  const int n = (int)b->h.size();
  std::vector<int> all, n1(n, 0), n2(n, 0);
  std::vector<double> tol1;
  std::vector<int> cap1;
  std::vector<char> stall1;
  for (int i = 0; i < n; ++i) {
    lgf_handle h = b->h[i];
    if (!h->loaded) return bfail(b, LGF_ERR_ARG, "member " + std::to_string(i) + " has no links loaded");
    cudaStreamSynchronize(h->stream);
    h->last_n32 = h->last_n64 = 0;
    all.push_back(i);
    const bool fp32 = h->mixed && h->cur == &h->e32;
    tol1.push_back(fp32 ? std::max(theta_tol, h->tail_theta) : theta_tol);
    int cap = max_iter;
    if (fp32 && h->tail_max32 >= 0 && h->tail_max32 < cap) cap = (int)h->tail_max32;
    cap1.push_back(cap);
    stall1.push_back(fp32 ? 1 : 0);
  }
  // phase 1: every member on its current engine (FP32 bulk, or FP64)
  int rc = run_members(b, all, tol1, cap1, stall1);
  if (rc) return rc;
  std::vector<int> tail;
  for (int i = 0; i < n; ++i) {
    lgf_handle h = b->h[i];
    n1[i] = h->st_host->iters;
    h->total_updates += n1[i];
    if (h->mixed && h->cur == &h->e32) {
      h->last_n32 = n1[i];
      if (h->st_host->theta < theta_tol) continue;
      // FP64 tail from the loaded links and the reunitarised accumulated G
      cudaStream_t saved = h->stream;
      h->stream = b->main;
      rc = queue_tail_start(h);
      h->stream = saved;
      if (rc) return bfail(b, rc, h->err);
      tail.push_back(i);
    } else {
      h->last_n64 = n1[i];
    }
  }
  LGF_BCUDA(b, cudaStreamSynchronize(b->main));
  // phase 2: the FP64 tails together
  std::vector<double> tol2(tail.size(), theta_tol);
  std::vector<int> cap2;
  for (int i : tail) cap2.push_back(max_iter - n1[i] > 0 ? max_iter - n1[i] : 0);
  std::vector<char> stall2(tail.size(), 0);
  rc = run_members(b, tail, tol2, cap2, stall2);
  if (rc) return rc;
  LGF_BCUDA(b, cudaStreamSynchronize(b->main));
  for (int i : tail) {
    n2[i] = b->h[i]->st_host->iters;
    b->h[i]->last_n64 = n2[i];
    b->h[i]->total_updates += n2[i];
  }
  bool all_conv = true;
  for (int i = 0; i < n; ++i) {
    const bool conv = b->h[i]->st_host->theta < theta_tol;
    all_conv = all_conv && conv;
    if (iters_out) iters_out[i] = n1[i] + n2[i];
    if (converged_out) converged_out[i] = conv ? 1 : 0;
  }
  return all_conv ? LGF_OK : bfail(b, LGF_ERR_NOT_CONVERGED, "some members reached max_iter with theta >= tol");
}

const char* lgf_batch_last_error(lgf_batch b) { return b ? b->err.c_str() : ""; }

int lgf_batch_autotune(lgf_batch b, int reps, int* lanes_out) {
  if (!b || reps < 1) return LGF_ERR_ARG;
  const int n = (int)b->h.size();
  std::vector<int> all;
  for (int i = 0; i < n; ++i) {
    if (!b->h[i]->loaded) return bfail(b, LGF_ERR_ARG, "member " + std::to_string(i) + " has no links loaded");
    cudaStreamSynchronize(b->h[i]->stream);
    all.push_back(i);
  }
  std::vector<double> tol(n, -1.0);
  std::vector<int> cap(n, reps);
  std::vector<char> nostall(n, 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return bfail(b, LGF_ERR_CUDA, "event creation failed");
  }
  const int cands[] = {1, 2, 4, 8, 16, 0};
  int best = 0, rc = LGF_OK;
  float best_ms = INFINITY;
  const int saved = b->lanes;
  for (int c : cands) {
    if (c > n) continue;
    b->lanes = c;
    std::vector<unsigned long long> conds;
    rc = capture(b, all, conds);
    if (rc) break;
    for (int pass = 0; pass < 2 && !rc; ++pass) {  // a warm-up launch, then the timed one
      rc = reset_members(b, all, tol, cap, nostall, conds);
      if (rc) break;
      cudaEventRecord(e0, b->main);
      if (cudaGraphLaunch(b->exec, b->main) != cudaSuccess) rc = bfail(b, LGF_ERR_CUDA, "graph launch failed");
      cudaEventRecord(e1, b->main);
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = bfail(b, LGF_ERR_CUDA, "graph launch failed");
      for (int i : all) b->h[i]->total_updates += reps;  // the tuning updates are applied
    }
    if (rc) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(b);
  if (rc) {
    b->lanes = saved;
    return rc;
  }
  b->lanes = best;
  if (lanes_out) *lanes_out = best;
  return LGF_OK;
}

int lgf_batch_set_lanes(lgf_batch b, int lanes) {
  if (!b || lanes < 0) return LGF_ERR_ARG;
  if (lanes != b->lanes) drop_graph(b);
  b->lanes = lanes;
  return LGF_OK;
}

int lgf_net_param_count(void) { return warm::kParams; }

int lgf_net_create(unsigned long long seed, lgf_net* out) {
  if (!out) return LGF_ERR_ARG;
  *out = nullptr;
  lgf_net_ctx* n = new (std::nothrow) lgf_net_ctx();
  if (!n) return nfail(nullptr, LGF_ERR_OOM, "host allocation failed");
  if (cudaGetDevice(&n->device) != cudaSuccess) {
    delete n;
    return nfail(nullptr, LGF_ERR_CUDA, "no CUDA device");
  }
  const size_t P = warm::kParams;
  n->p = static_cast<float*>(net_alloc(n, P * 4));
  n->m = static_cast<float*>(net_alloc(n, P * 4));
  n->v = static_cast<float*>(net_alloc(n, P * 4));
  n->g = static_cast<float*>(net_alloc(n, P * 4));
  n->W1 = net_alloc(n, (size_t)kW1 * 2);
  n->W2 = net_alloc(n, (size_t)kW2 * 2);
  n->W3 = net_alloc(n, (size_t)81 * 32 * 16 * 2);
  n->Wt1 = net_alloc(n, (size_t)kW1 * 2);
  n->Wt2 = net_alloc(n, (size_t)kW2 * 2);
  n->Wt3 = net_alloc(n, (size_t)81 * 32 * 16 * 2);
  n->tc_err = static_cast<int*>(net_alloc(n, 2 * sizeof(int)));
  n->b1 = static_cast<float*>(net_alloc(n, 32 * 4));
  n->b2 = static_cast<float*>(net_alloc(n, 32 * 4));
  n->b3 = static_cast<float*>(net_alloc(n, 16 * 4));
  n->gW3p = static_cast<float*>(net_alloc(n, (size_t)81 * 32 * 16 * 4));
  n->gb3p = static_cast<float*>(net_alloc(n, 16 * 4));
  if (!n->p || !n->m || !n->v || !n->g || !n->W1 || !n->W2 || !n->W3 || !n->b1 || !n->b2 || !n->b3 || !n->gW3p ||
      !n->gb3p || !n->Wt1 || !n->Wt2 || !n->Wt3 || !n->tc_err) {
    std::string msg = "device allocation of the network failed";
    lgf_net_destroy(n);
    return nfail(nullptr, LGF_ERR_OOM, msg);
  }
  const int err_init[2] = {0, warm::kConvWaitPolls};
  if (cudaMemcpy(n->tc_err, err_init, sizeof err_init, cudaMemcpyHostToDevice) != cudaSuccess) {
    lgf_net_destroy(n);
    return nfail(nullptr, LGF_ERR_CUDA, "initialising the network's error flag failed");
  }
  // He-normal initialisation; the last layer 100x smaller so that g0 starts
  // close to the identity (the warm start starts as "no warm start")
  std::vector<float> hp(P, 0.0f);
  const double s1 = sqrt(2.0 / (81.0 * 48)), s2 = sqrt(2.0 / (81.0 * 32)), s3 = 0.01 * sqrt(1.0 / (81.0 * 32));
  for (int i = 0; i < kW1; ++i) hp[i] = (float)(s1 * normal_at(seed, i));
  for (int i = 0; i < kW2; ++i) hp[kOW2 + i] = (float)(s2 * normal_at(seed, kOW2 + i));
  for (int i = 0; i < kW3; ++i) hp[kOW3 + i] = (float)(s3 * normal_at(seed, kOW3 + i));
  int rc = lgf_net_set_params(n, hp.data());
  if (rc) {
    std::string msg = n->err;
    lgf_net_destroy(n);
    return nfail(nullptr, rc, msg);
  }
  *out = n;
  return LGF_OK;
}

int lgf_net_destroy(lgf_net n) {
  if (!n) return LGF_ERR_ARG;
  cudaDeviceSynchronize();
  while (!n->allocs.empty()) net_free(n, n->allocs.back().first);
  delete n;
  return LGF_OK;
}

int lgf_net_get_params(lgf_net n, float* host) {
  if (!n || !host) return LGF_ERR_ARG;
  LGF_NCUDA(n, cudaMemcpy(host, n->p, (size_t)warm::kParams * 4, cudaMemcpyDeviceToHost));
  return LGF_OK;
}

int lgf_net_set_wait_budget(lgf_net n, long long polls) {
  if (!n) return LGF_ERR_ARG;
  const int v = polls < 0 ? warm::kConvWaitPolls : (int)(polls < warm::kConvWaitPolls ? polls : warm::kConvWaitPolls);
  LGF_NCUDA(n, cudaDeviceSynchronize());
  LGF_NCUDA(n, cudaMemcpy(n->tc_err + 1, &v, sizeof v, cudaMemcpyHostToDevice));
  return LGF_OK;
}

int lgf_net_set_params(lgf_net n, const float* host) {
  if (!n || !host) return LGF_ERR_ARG;
  const size_t P = warm::kParams;
  LGF_NCUDA(n, cudaMemcpy(n->p, host, P * 4, cudaMemcpyHostToDevice));
  LGF_NCUDA(n, cudaMemset(n->m, 0, P * 4));
  LGF_NCUDA(n, cudaMemset(n->v, 0, P * 4));
  n->step = 0;
  int rc = net_pack(n, nullptr);
  if (rc) return rc;
  LGF_NCUDA(n, cudaDeviceSynchronize());
  return LGF_OK;
}

int lgf_net_forward(lgf_net n, lgf_handle h, float* host_c) {
  int rc = net_check_handle(n, h);
  if (!rc) rc = net_forward(n, h);
  if (rc) return rc;
  if (host_c) {
    // [V][16] FP32 on the device -> [V][8] on the host
    LGF_NCUDA(n, cudaMemcpy2DAsync(host_c, 8 * sizeof(float), n->c, 16 * sizeof(float), 8 * sizeof(float),
                                   (size_t)h->V, cudaMemcpyDeviceToHost, h->stream));
  }
  LGF_NCUDA(n, cudaStreamSynchronize(h->stream));
  return net_check_tc(n);
}

int lgf_net_train_step(lgf_net n, lgf_handle h, double lr, double* F_out, float* host_grad) {
  int rc = net_check_handle(n, h);
  if (!rc) rc = net_forward(n, h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  const int V = (int)h->V;
  // g0 and the gradient of the transformed links (gauge representation, G = g0)
  LGF_NCUDA(n, warm::launch_expmap(h->e32.nc, n->c, 16, n->G0, V, s));
  rc = reset_state(h, -1.0, 0, false);
  if (rc) return nfail(n, rc, h->err);
  LGF_NCUDA(n, launch_gradient_grep(h->e32.nc, h->e32.U, n->G0, h->e32.D, h->partial, h->geo, h->st, 0, s));
  LGF_NCUDA(n, warm::launch_signal(h->e32.D, V, (float)(-1.0 / (24.0 * (double)V)), n->gc, s));
  const size_t P = warm::kParams;
  LGF_NCUDA(n, cudaMemsetAsync(n->g, 0, P * 4, s));
  LGF_NCUDA(n, cudaMemsetAsync(n->gW3p, 0, (size_t)81 * 32 * 16 * 4, s));
  LGF_NCUDA(n, cudaMemsetAsync(n->gb3p, 0, 16 * 4, s));
  // layer 3 (a2 -> c)
  LGF_NCUDA(n, warm::launch_conv_bwd_weight(3, n->a2, n->gc, n->gW3p, h->geo, s));
  LGF_NCUDA(n, warm::launch_bias_grad(16, n->gc, n->gb3p, V, s));
  LGF_NCUDA(n, warm::launch_conv_bwd_data_tc(3, n->gc, n->W3, n->a2, n->ga2, h->geo, n->tc_err, s));
  // layer 2 (a1 -> a2)
  LGF_NCUDA(n, warm::launch_conv_bwd_weight(2, n->a1, n->ga2, n->g + kOW2, h->geo, s));
  LGF_NCUDA(n, warm::launch_bias_grad(32, n->ga2, n->g + kOB2, V, s));
  LGF_NCUDA(n, warm::launch_conv_bwd_data_tc(2, n->ga2, n->W2, n->a1, n->ga1, h->geo, n->tc_err, s));
  // layer 1 (x0 -> a1)
  LGF_NCUDA(n, warm::launch_conv_bwd_weight(1, n->x0, n->ga1, n->g, h->geo, s));
  LGF_NCUDA(n, warm::launch_bias_grad(32, n->ga1, n->g + kOB1, V, s));
  LGF_NCUDA(n, warm::launch_unpad_grad3(n->gW3p, n->gb3p, n->g + kOW3, n->g + kOB3, s));
  h->launches += 14;
  if (host_grad) LGF_NCUDA(n, cudaMemcpyAsync(host_grad, n->g, P * 4, cudaMemcpyDeviceToHost, s));
  if (lr > 0.0) {
    n->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)n->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)n->step)));
    LGF_NCUDA(n, warm::launch_adam(n->p, n->g, n->m, n->v, (int)P, (float)lr, (float)b1, (float)b2, c1, c2, 1e-12f, s));
    rc = net_pack(n, s);
    if (rc) return rc;
    h->launches += 2;
  }
  rc = sync_state(h);
  if (rc) return nfail(n, rc, h->err);
  rc = net_check_tc(n);
  if (rc) return rc;
  if (F_out) *F_out = h->st_host->F;
  return LGF_OK;
}

int lgf_net_warm_start(lgf_net n, lgf_handle h) {
  int rc = net_check_handle(n, h);
  if (rc) return rc;
  if (h->total_updates != 0) return nfail(n, LGF_ERR_ARG, "apply the warm start right after lgf_load_links");
  rc = net_forward(n, h);
  if (rc) return rc;
  LGF_NCUDA(n, warm::launch_expmap(h->e32.nc, n->c, 16, h->G, (int)h->V, h->stream));
  h->launches += 1;
  LGF_NCUDA(n, cudaStreamSynchronize(h->stream));
  return net_check_tc(n);
}

int lgf_net_conv(lgf_net n, int layer, int backward, const void* in, const void* mask, void* out, float* out_f32,
                 int Lx, int Ly, int Lz, int Lt, void* stream) {
  if (!n) return LGF_ERR_ARG;
  if (layer < 1 || layer > 3 || (backward != 0 && backward != 1) || (backward && layer == 1))
    return nfail(n, LGF_ERR_ARG, "lgf_net_conv: layer 1..3 forward, 2..3 backward");
  if (!in || !out) return nfail(n, LGF_ERR_ARG, "lgf_net_conv: in and out must be device pointers");
  Geom geo{};
  const int Ls[4] = {Lx, Ly, Lz, Lt};
  int64_t V = 1;
  for (int a = 0; a < 4; ++a) {
    if (Ls[a] < 2 || Ls[a] > kMaxL) return nfail(n, LGF_ERR_ARG, "lgf_net_conv: each extent must be in [2, 64]");
    geo.L[a] = Ls[a];
    geo.stride[a] = V;
    V *= Ls[a];
  }
  geo.V = V;
  geom_init_rcp(geo);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* const Wt[3] = {n->Wt1, n->Wt2, n->Wt3};
  void* const W[3] = {n->W1, n->W2, n->W3};
  const float* const b[3] = {n->b1, n->b2, n->b3};
  if (!backward)
    LGF_NCUDA(n, warm::launch_conv_fwd_tc(layer, in, Wt[layer - 1], b[layer - 1], out, out_f32, geo, n->tc_err, s));
  else
    LGF_NCUDA(n, warm::launch_conv_bwd_data_tc(layer, in, W[layer - 1], mask, out, geo, n->tc_err, s));
  LGF_NCUDA(n, cudaStreamSynchronize(s));
  return net_check_tc(n);
}

const char* lgf_net_last_error(lgf_net n) { return n ? n->err.c_str() : g_last_create_error.c_str(); }

int lgf_history(lgf_handle h, double* theta_out, int cap, int* n_out) {
  if (!h) return LGF_ERR_ARG;
  const int n = h->hist_n < cap ? h->hist_n : cap;
  if (theta_out && n > 0) LGF_CUDA(h, cudaMemcpy(theta_out, h->hist, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
  if (n_out) *n_out = n;
  return LGF_OK;
}

int lgf_profile(lgf_handle h, int enable) {
  if (!h) return LGF_ERR_ARG;
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (enable) {
    h->ev_kind.clear();
    for (int k = 0; k < LGF_NUM_KERNELS; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_n[k] = 0;
    }
  }
  h->profiling = enable != 0;
  return LGF_OK;
}

int lgf_profile_read(lgf_handle h, double* ms, long long* launches, int n) {
  if (!h || n < 0) return LGF_ERR_ARG;
  LGF_CUDA(h, cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < h->ev_kind.size(); ++i) {
    float t = 0.0f;
    LGF_CUDA(h, cudaEventElapsedTime(&t, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
    h->prof_ms[h->ev_kind[i]] += t;
    h->prof_n[h->ev_kind[i]] += 1;
  }
  h->ev_kind.clear();
  for (int k = 0; k < n && k < LGF_NUM_KERNELS; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_n[k];
  }
  return LGF_OK;
}

const char* lgf_kernel_name(int kind) {
  static const char* names[LGF_NUM_KERNELS] = {"gradient", "fft_axis",   "fft_xy", "fft_zt", "build_g",
                                               "update",   "accumulate", "other",  "fft_t",  "xy_gstep"};
  return (kind >= 0 && kind < LGF_NUM_KERNELS) ? names[kind] : "";
}

const char* lgf_last_error(lgf_handle h) { return h ? h->err.c_str() : g_last_create_error.c_str(); }

long long lgf_launch_count(lgf_handle h) { return h ? h->launches : -1; }

}  // extern "C"
