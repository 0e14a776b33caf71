// Host-side launchers of the liblgf kernels (one translation unit each for
// the link kernels and the FFT kernels; the C ABI lives in lgf_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lgf_common.cuh"

namespace lgf {

// Launch with programmatic stream serialization: the kernel's launch overlaps
// the previous kernel's drain; the kernel must begin with pdl_wait().
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace lgf

namespace lgf {

constexpr int kMaxL = 64;       // longest lattice extent the on-chip FFT takes
constexpr int kMaxStages = 6;   // radix stages per axis (4^3 = 64)

// Mixed-radix factorisation of one axis, radix 4 first, then 2, 3, 5.
struct AxisPlan {
  int L;
  int nst;
  int radix[kMaxStages];
};

// Everything the FFT kernels need to know about the lattice.
struct FftGeom {
  AxisPlan ax[4];
  int L[4];
  int64_t V;
  double p2max;   // sum_mu max_k 4 sin^2(pi k / L_mu)
  int Bx;         // consecutive x per z-t CTA
  int Pxy;        // padded row pitch of an x-y plane in shared memory
  int Pt;         // padded pitch of one t slice of a z-t tile
};

bool make_axis_plan(int L, AxisPlan* p);

// byte sizes of the dynamic shared memory each FFT kernel needs
size_t fft_xy_smem(const FftGeom& fg, int real_bytes);
size_t fft_zt_smem(const FftGeom& fg, int real_bytes);
cudaError_t fft_set_smem_limits(int real_bytes, size_t xy, size_t zt);

// prec: 8 = FP64, 4 = FP32; nc: complex entries stored per matrix (9 or 6)
// gradient + FP64 F/theta reduction (its last block finishes it); mode 0: F
// and theta only, mode 1: also the stop decision of an iteration queue
cudaError_t launch_gradient(int prec, int nc, const void* U, void* D, double2* partial,
                            const Geom& geo, DevState* st, int mode, cudaStream_t s);
cudaError_t launch_fft_xy(int prec, void* D, const FftGeom& fg, const void* tw, int inverse,
                          const DevState* st, cudaStream_t s);
cudaError_t launch_fft_zt(int prec, void* D, const FftGeom& fg, const void* tw,
                          const double* sin2, const DevState* st, cudaStream_t s);
// exact: g from the exact exponential of alpha/2 Delta~ instead of 1 + alpha/2 Delta~
cudaError_t launch_build_g(int prec, int nc, const void* D, void* g, int64_t V, double half_alpha,
                           bool reunit_fp64, bool exact, const DevState* st, cudaStream_t s);
cudaError_t launch_update(int prec, int nc, void* U, const void* g, const Geom& geo,
                          const DevState* st, cudaStream_t s);
// host [s][mu][3][3] complex128 layout (on the device) <-> SoA storage
// (nmu matrices per site: 4 for links, 1 for a gauge field)
cudaError_t launch_aos_to_soa(int prec, int nc, const double* aos, void* U, int64_t V, int nmu, cudaStream_t s);
// host-layout link load/store staged through shared memory (k_links.cu); the
// AoS pointer may be host memory the device can access (16-byte aligned).
// Load: nc64 (9 or 6, FP64) and nc32 (9, 6 or 0, FP32) SoA outputs from one read.
constexpr int kStageMats = 256;   // links per CTA
constexpr int kStagePitch = 19;   // doubles per staged link
cudaError_t launch_load_aos(int nc64, int nc32, const double* aos, void* U64, void* U32, int64_t V, cudaStream_t s);
cudaError_t launch_store_aos(int prec, int nc, const void* U, double* aos, int64_t V, cudaStream_t s);
cudaError_t launch_soa_to_aos(int prec, int nc, const void* U, double* aos, int64_t V, int nmu, cudaStream_t s);
// G <- reunitarised g G (storage precision); FP64 reunitarised copy of G
cudaError_t launch_accumulate(int prec, int nc, void* G, const void* g, int64_t V, const DevState* st,
                              cudaStream_t s);
// double-float links (hi planes, then lo planes) -> AoS doubles (host or device); with eta (not
// null) the tail's links (1 + eta) Udf (1 + eta(x+mu))^dag
cudaError_t launch_store_aos_df(const void* Udf, const void* eta, const Geom& geo, double* aos, cudaStream_t s);
cudaError_t launch_promote_gauge(int prec, int nc, const void* G, void* out64, int64_t V, cudaStream_t s);
// G <- 1 at every site
cudaError_t launch_set_identity(int prec, int nc, void* G, int64_t V, cudaStream_t s);
// packed gradient fields [4][V] -> [V][4] complex128 (for probes)
cudaError_t launch_unpack_fields(int prec, const void* D, double* out, int64_t V, cudaStream_t s);

// per-axis register FFT passes (k_fft_axis.cu); lengths 4..32 (FP64) and up
// to 64 (FP32) with radices 4, 2, 3, 5
bool axis_pass_supported(int prec, int L);
cudaError_t axis_pass_init();
cudaError_t launch_xpass(int prec, int L, void* D, int64_t V, int inverse, const DevState* st, cudaStream_t s);
cudaError_t launch_strided(int prec, int L, void* D, int64_t V, int64_t S, int inverse, const DevState* st,
                           cudaStream_t s);
// FP64: factor from the per-site table kfac; FP32: from s2p[axis][position]
// (4 sin^2 at the digit-reversed frequency) and c_over_V = p2_max / V
cudaError_t launch_tpass(int prec, int L, void* D, int64_t V, int Lx, int Ly, const void* kfac, const float* s2p,
                         float c_over_V, const DevState* st, cudaStream_t s);

// three-pass plane pipeline with register FFTs: x-y plane (Lx = Ly) kernels
// (k_fft_plane.cu) and z-t plane (fwd, acceleration factor, inv) kernels
// (k_fft_zt.cu) for a list of instantiated shapes
#define LGF_ZT_F32(X)                                                                                      \
  X(4, 4) X(6, 6) X(8, 8) X(12, 12) X(16, 16) X(20, 20) X(24, 24) X(32, 32) X(48, 48) X(48, 8) X(48, 12) \
  X(24, 48) X(32, 8) X(32, 16) X(16, 32)
#define LGF_ZT_F64(X) \
  X(4, 4) X(6, 6) X(8, 8) X(12, 12) X(16, 16) X(20, 20) X(24, 24) X(32, 32) X(32, 8) X(32, 16) X(16, 32)
bool plane_pipeline_supported(int prec, int Lx, int Ly, int Lz, int Lt);
cudaError_t plane_pipeline_init();
cudaError_t plane_zt_init();
cudaError_t launch_plane_xy(int prec, int L, void* D, int64_t V, int Lz, int Lt, int inverse, const DevState* st,
                            cudaStream_t s);
// z-t pass schedule: bx = x-run width of a tile (0: the default, 4 FP32 / 2
// FP64; or twice that), ro = radix order of the z and t transforms (0, or 1
// for FP32 where it changes the stages); s2p holds [2][4][kMaxL] FP32 factors
bool plane_zt_schedule_supported(int prec, int Lx, int Lz, int Lt, int bx, int ro);
cudaError_t launch_plane_zt(int prec, int Lx, int Ly, int Lz, int Lt, void* D, const void* kfac, const float* s2p,
                            float c_over_V, int bx, int ro, const DevState* st, cudaStream_t s);
// inverse x-y pass fused with G <- g G (FP32 gauge representation; Lx = Ly
// one of 4, 6, 8, 12, 16, 20, 24, 32)
bool plane_xyinv_gstep_supported(int prec, int L);
// the double-float tail's inverse x-y pass fused with its eta step (FP32
// packed gradient, Lx = Ly one of 4, 6, 8, 12, 16, 20, 24, 32)
bool plane_xyinv_eta_supported(int L);
cudaError_t plane_xyinv_eta_init();
cudaError_t launch_plane_xyinv_eta(int L, const void* D, void* eta, int64_t V, int Lz, int Lt, double half_alpha,
                                   const DevState* st, cudaStream_t s);
cudaError_t launch_plane_xyinv_gstep(int L, int nc, const void* D, void* G, int64_t V, int Lz, int Lt,
                                     double half_alpha, bool reunit_fp64, const DevState* st, cudaStream_t s);

// FP32 engine in gauge representation (k_gauge_rep.cu): links formed on the
// fly as G U0 G^dagger; the update acts on G
cudaError_t launch_gradient_grep(int nc, const void* U0, const void* G, void* D, double2* partial, const Geom& geo,
                                 DevState* st, int mode, cudaStream_t s);
cudaError_t launch_gstep(int nc, const void* D, void* G, void* g_out, int64_t V, double half_alpha, bool reunit_fp64,
                         bool exact, const DevState* st, cudaStream_t s);
cudaError_t launch_materialize(int nc, const void* U0, const void* G, double* aos, const Geom& geo, cudaStream_t s);

// FP64 tail by defect correction with double-float links (k_tail.cu): Udf
// holds 36 V complex hi parts followed by 36 V complex lo parts
// G (FP32, rows 0-1 used) -> Gh, Gl (2 x 9 FP32 complex planes), reunitarised in double-float
// (1 + eta)(Gh + Gl) of a double-float tail as FP64 [s][3][3] complex (device
// memory, or host memory the device writes directly)
cudaError_t launch_store_gauge_df(const void* g_df, const void* eta, int64_t V, double* out, cudaStream_t s);
cudaError_t launch_promote_df(const void* G32, void* g_df, int64_t V, cudaStream_t s);
// Udf = Gh+Gl U_loaded (Gh+Gl)(x+mu)^dag in double-float (hi planes, then lo planes)
cudaError_t launch_tail_start_df(const void* Uin64, const void* g_df, void* Udf, const Geom& geo, cudaStream_t s);
// the tail in gauge representation: links (1 + eta) Udf (1 + eta(x+mu))^dag, eta in double-float
// (9 complex hi planes, then 9 lo planes; the gradient reads the hi planes)
// the fixed part of the tail's gradient: Delta(Udf) packed (4 V complex FP32), then each site's
// F term sum_mu Re tr Udf_mu(x) in double-float (V float pairs); 40 bytes per site in base
cudaError_t launch_tail_base(const void* Udf, void* base, const Geom& geo, cudaStream_t s);
cudaError_t launch_gradient_tail_eta(const void* Udf, const void* eta, const void* base, void* D32,
                                     double2* partial, const Geom& geo, DevState* st, int mode, cudaStream_t s);
// eta <- (1 + eps)(1 + eta) - 1, eps = X + X^2/2 with X = half_alpha Delta~ from D32
cudaError_t launch_tail_eta_step(const void* D32, void* eta, int64_t V, double half_alpha, const DevState* st,
                                 cudaStream_t s);
// Udf <- (1 + eta) Udf (1 + eta(x+mu))^dag, then eta <- 0
cudaError_t launch_tail_apply_eta(void* Udf, void* eta, const Geom& geo, cudaStream_t s);
cudaError_t launch_df_to_fp64(const void* Udf, void* U64, int64_t V, cudaStream_t s);
// FP64 tail by defect correction (k_tail.cu): FP64 links, FP32 FFT and step
cudaError_t launch_gradient_tail(const void* U64, void* D32, double2* partial, const Geom& geo, DevState* st,
                                 int mode, cudaStream_t s);
cudaError_t launch_tail_step(const void* D32, void* eps, int64_t V, double half_alpha, const DevState* st,
                             cudaStream_t s);
cudaError_t launch_tail_update(void* U64, const void* eps, const Geom& geo, const DevState* st, cudaStream_t s);

// learned warm start (k_warm.cu): features, BF16 tensor-core convolutions,
// exp map, training signal, Adam
namespace warm {
constexpr int kParams = 81 * 48 * 32 + 32 + 81 * 32 * 32 + 32 + 81 * 32 * 8 + 8;
cudaError_t launch_features(int nc, const void* U0, void* x, const Geom& geo, cudaStream_t s);
cudaError_t launch_expmap(int nc, const float* c, int ldc, void* G, int V, cudaStream_t s);
cudaError_t launch_signal(const void* D, int V, float coef, void* gc, cudaStream_t s);
cudaError_t launch_conv_bwd_weight(int layer, const void* x, const void* gy, float* gW, const Geom& geo,
                                   cudaStream_t s);
cudaError_t launch_bias_grad(int co, const void* gy, float* gb, int V, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float c1,
                        float c2, float eps, cudaStream_t s);
cudaError_t launch_pack_weights(const float* p, void* W1, void* W2, void* W3, float* b1, float* b2, float* b3,
                                void* Wt1, void* Wt2, void* Wt3, cudaStream_t s);
// tcgen05 implicit-GEMM convolutions (forward and backward data); err[0] is
// set to 1 if a bounded wait inside a CTA expired; err[1] is the poll budget
// of the stage waits (kConvWaitPolls by default)
constexpr int kConvWaitPolls = 1 << 22;
cudaError_t launch_conv_fwd_tc(int layer, const void* x, const void* Wt, const float* b, void* y, float* yf,
                               const Geom& geo, int* err, cudaStream_t s);
cudaError_t launch_conv_bwd_data_tc(int layer, const void* gy, const void* W, const void* a, void* gx,
                                    const Geom& geo, int* err, cudaStream_t s);
cudaError_t launch_unpad_grad3(const float* gW3p, const float* gb3p, float* gW3, float* gb3, cudaStream_t s);
}  // namespace warm

// text returned by lgf_last_error(NULL) on this host thread
void set_global_error(const std::string& msg);

constexpr int kGradThreads = 256;  // k_gradient block size
constexpr int kGrepThreads = 256;  // k_gradient_grep block size
inline int gradient_blocks(int64_t V) { return (int)((V + kGradThreads - 1) / kGradThreads); }
// capacity of the block-partials buffer: enough for the smallest block size
inline int64_t partial_capacity(int64_t V) { return (V + 63) / 64 + 1; }

}  // namespace lgf
