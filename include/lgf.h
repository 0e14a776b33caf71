/*
 * lgf.h -- C ABI of liblgf: SU(3) lattice Landau gauge fixing by steepest
 * descent with Fourier acceleration on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one the paper uses (Cardoso, Bicudo, Silva, Oliveira,
 * "Landau Gauge Fixing on GPUs and String Tension", Sec. 1: steepest descent
 * with Fourier acceleration after Davies et al.; Sec. 2.2: one thread per
 * site, structure-of-arrays lattice, 4D FFT built from 2D plus 2D
 * transforms).  The paper prints no formula of the iteration; the library
 * computes, per iteration and on a periodic lattice L = (Lx, Ly, Lz, Lt) of
 * V sites:
 *
 *   A(x)      = sum_mu [U_mu(x - mu) - U_mu(x)]
 *   Delta(x)  = A - A^dagger - (1/3) Tr(A - A^dagger)          (gradient)
 *   F         = 1/(4*3*V) sum_{x,mu} Re Tr U_mu(x)              (functional)
 *   theta     = 1/(3*V)   sum_x Tr Delta Delta^dagger           (convergence)
 *   Delta~    = FFT^-1[ p2_max / p2(k) * FFT[Delta] ], 0 at k = 0,
 *               p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu)
 *   g(x)      = reunitarised (1 + alpha/2 Delta~(x))             (gauge step;
 *               reunitarised exp(alpha/2 Delta~(x)) with LGF_EXP_ORDER = 0)
 *   U_mu(x)  <- g(x) U_mu(x) g(x + mu)^dagger                    (update)
 *
 * theta and F always describe the links *before* an update; an iteration is
 * one applied update.
 *
 * Conventions for every entry point:
 *   - Return value: LGF_OK (0) or a negative lgf_status.  No exception,
 *     abort or device trap leaves the library; lgf_last_error() gives text.
 *   - Host link arrays are complex128 "array of structures" in the order
 *     [s][mu][i][j] (re, im interleaved), s = x + Lx*(y + Ly*(z + Lz*t)),
 *     mu = 0..3 = x, y, z, t: V*4*18 doubles.  They are caller-owned and
 *     copied; the library keeps no pointer to them.
 *   - Device memory is library-owned, obtained through the allocator set
 *     with lgf_set_allocator() (cudaMalloc by default) on the device that was
 *     current at lgf_create().  All work runs on the handle's stream (the
 *     legacy default stream until lgf_set_stream()).  Every call that
 *     computes returns after its work on that stream has finished.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef LGF_H
#define LGF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgf_ctx* lgf_handle;

/* Storage / arithmetic of the working links (paper Sec. 3.1 compares single
 * and double precision and the 18-real and 12-real forms). */
enum lgf_dtype {
  LGF_F64 = 0,      /* FP64 links, 18 reals, FP64 everywhere                  */
  LGF_F32 = 1,      /* FP32 links/FFT/update, 18 reals; FP64 F, theta sums     */
  LGF_F32_R12 = 2,  /* as LGF_F32, links stored as rows 1-2 (12 reals), row 3
                       rebuilt as conj(row1 x row2) on load (paper Sec. 2.2)  */
  LGF_F64_R12 = 3   /* FP64, 12-real storage                                  */
};

enum lgf_status {
  LGF_OK = 0,
  LGF_ERR_ARG = -1,            /* bad argument / unsupported lattice           */
  LGF_ERR_CUDA = -2,           /* a CUDA runtime call failed                    */
  LGF_ERR_OOM = -3,            /* the allocator returned NULL                   */
  LGF_ERR_NOT_CONVERGED = -4,  /* lgf_fix used max_iter updates, theta >= tol   */
  LGF_ERR_NONFINITE = -5,      /* F or theta became NaN/Inf (bad input links)   */
  LGF_ERR_TIMEOUT = -6         /* a bounded device wait gave up                 */
};

enum lgf_param {
  LGF_ALPHA = 0,        /* step size alpha (default 0.08)                       */
  LGF_CHECK_EVERY = 1,  /* lgf_fix under lgf_profile: at most this many iterations
                           queued between host checks (32).  Without profiling
                           each phase is one device-side graph loop.          */
  LGF_TAIL_THETA = 2,   /* mixed precision: theta at which the FP32 phase hands
                           over to the FP64 tail (default 1e-12, just above
                           where FP32 rounding stalls the FP32 phase)          */
  LGF_TAIL_MAX_FP32 = 3, /* mixed precision: cap on FP32 iterations (default: all) */
  LGF_REUNIT_FP64 = 4,   /* FP32 storage: reunitarise g in FP64 arithmetic (0/1,
                            default 0: g is stored in FP32, so FP64 arithmetic
                            would be rounded away on the store)                */
  LGF_FFT_PIPELINE = 5,  /* FFT pipeline: 0 (default) automatic -- register
                            planes (x-y + z-t passes) where instantiated, else
                            per-axis register passes, else shared-memory
                            Stockham planes; 1 Stockham planes; 2 per-axis
                            passes; 3 register planes (1 where not available) */
  LGF_TAIL_MODE = 7,     /* mixed precision: 0 (default) finishes with the
                            defect-correction tail when the FP32 phase reached
                            theta < 1e-8: FP32 acceleration and step, g = 1 +
                            eps with eps the exponential to second order, the
                            correction added to links held in double-float
                            form (FP32 hi + lo, 48 bits), which they keep
                            until the next load (lgf_store_links writes them
                            as FP64, hi + lo); 2 the same tail on FP64 links;
                            1 always uses the plain FP64 iteration.  Values
                            other than 0, 1, 2 give LGF_ERR_ARG.              */
  LGF_TRACK_G = 9,       /* FP64 handles, from the next load: 1 accumulates the
                            gauge transformation G(x) <- reunitarised g(x) G(x)
                            with every update, so that lgf_store_gauge can
                            return it (one more SU(3) field in FP64 and one
                            more kernel per iteration); 0 (default) does not.
                            Mixed-precision handles always keep it (their FP32
                            phase works on G); the parameter has no effect
                            there.                                              */
  LGF_EXP_ORDER = 8,     /* g from the accelerated gradient (paper Sec. 1, the
                            cited steepest descent: g = exp(alpha/2 Delta~)):
                            1 (default) reunitarised 1 + alpha/2 Delta~, the
                            first-order form; 0 the reunitarised exact
                            exponential, by a Taylor series with scaling and
                            squaring (degree 16 in FP64, 9 in FP32 arithmetic).
                            Both fix the same gauge.  With 0 the FP32 gauge
                            step runs unfused from the inverse transform; the
                            FP64 defect tail always uses 1 + eps, eps the
                            exponential to second order, which equals the
                            exact one to FP64 rounding at the tail's steps
                            (|alpha/2 Delta~| < 1e-5).  Other values give
                            LGF_ERR_ARG.                                        */
  LGF_LINK_UPDATE = 6    /* FP32 storage, from the next load: 0 (default) keeps
                            the loaded links and applies each update to the
                            accumulated gauge transformation G, forming
                            G U G^dagger on the fly; 1 updates the FP32 links
                            in place and accumulates G beside them            */
};

/* Device allocator hooks.  alloc returns a device pointer (NULL on failure);
 * free releases it.  Passing NULL for both restores cudaMalloc/cudaFree.
 * Process-wide; affects handles created afterwards. */
typedef void* (*lgf_alloc_fn)(size_t bytes, int device, void* stream, void* user);
typedef void (*lgf_free_fn)(void* ptr, size_t bytes, int device, void* stream, void* user);
int lgf_set_allocator(lgf_alloc_fn alloc, lgf_free_fn free_fn, void* user);

/* Create a context for an Lx x Ly x Lz x Lt periodic lattice.  Paper Sec.
 * 2.2: one thread per lattice site, the site index rebuilt inside the kernel,
 * lattice constants in constant memory (here they live in the handle and are
 * passed by value to every kernel); Sec. 3.1: single or double precision,
 * 18-real or 12-real storage, the dtype choices here.  Each extent must be in [2, 64] and a
 * product of 2, 3 and 5 (the radices of the on-chip FFT); dtype is an
 * lgf_dtype.  Allocates all device buffers.  On failure *out is NULL and
 * lgf_last_error(NULL) describes the cause. */
int lgf_create(int Lx, int Ly, int Lz, int Lt, int dtype, lgf_handle* out);

/* Release every device buffer (after synchronising the handle's stream). */
int lgf_destroy(lgf_handle h);

/* Run subsequent work on this cudaStream_t (e.g. torch's current stream). */
int lgf_set_stream(lgf_handle h, void* cuda_stream);

/* Set a numeric parameter (lgf_param).  alpha must lie in (0, 0.125]: the
 * accelerated step contracts every mode by (1 - 16 alpha), which is stable
 * only for alpha < 1/8. */
int lgf_set_param(lgf_handle h, int key, double value);

/* Copy V*4*18 doubles of host links in (layout above), converting to the
 * handle's storage; links must be SU(3) to rounding.  Mixed-precision
 * handles also keep the FP64 input for the FP64 tail.
 * Paper Sec. 2.2: the lattice lives in global memory as a structure of
 * arrays, one plane per matrix element and direction, so that the FFT can
 * work on each element without reordering; the 12-real storage keeps rows 1
 * and 2 and rebuilds row 3 from unitarity.  This call performs that
 * re-layout (and, for LGF_F32*, the rounding to FP32) on the device. */
int lgf_load_links(lgf_handle h, const double* host_aos);

/* As lgf_load_links, from device memory (e.g. a torch tensor's data_ptr)
 * on the handle's device (paper Sec. 2.2, the same structure-of-arrays
 * re-layout).  dev_aos must hold V*4*18 doubles; it is read, not kept. */
int lgf_load_links_device(lgf_handle h, const double* dev_aos);

/* Copy the current links out, as V*4*18 host doubles (layout above).  12-real
 * storage rebuilds row 3 as conj(row1 x row2) (paper Sec. 2.2).  host_aos
 * is caller-owned; the call returns once it is written. */
int lgf_store_links(lgf_handle h, double* host_aos);

/* Copy out the gauge transformation G that the iterations since the last
 * load have applied, as V*18 host doubles ([s][i][j] complex, row-major):
 * the current links are G(x) U_mu(x) G(x+mu)^dagger of the loaded links U
 * (paper Sec. 1: gauge fixing searches the gauge orbit of the configuration;
 * G is the point of the orbit it reached, which fixes other fields to the
 * same gauge).  FP64 handles need LGF_TRACK_G set before the load; mixed
 * handles return G from their FP32 phase, or (1 + eta) G in FP64 after the
 * default double-float tail.  Returns LGF_ERR_ARG when the handle does not
 * hold it: an FP64 handle without LGF_TRACK_G, a mixed handle after an
 * FP64-link tail (LGF_TAIL_MODE 1 or 2, or a hand-over above theta = 1e-8),
 * or after lgf_probe on the double-float tail.  host_g is caller-owned; the
 * call returns once it is written. */
int lgf_store_gauge(lgf_handle h, double* host_g);

/* Apply exactly n iterations (no convergence test).  Mixed-precision handles
 * iterate in their FP32 storage.  One iteration is one step of the paper's
 * steepest descent with Fourier acceleration (Sec. 1, after Davies et al.),
 * with the gradient transformed as 2D plus 2D FFTs (Sec. 2.2): the formulas
 * at the top of this file, gradient through update.  n < 0 gives
 * LGF_ERR_ARG; n = 0 does nothing. */
int lgf_iterate(lgf_handle h, int n);

/* Fix to Landau gauge (paper Sec. 1: the singlet correlator is not gauge
 * invariant, so the links are first brought to Landau gauge by steepest
 * descent with Fourier acceleration; Sec. 3.1 measures that iteration in
 * single and double precision).
 * Iterate until theta < theta_tol or max_iter updates have been applied.
 * *iters_out (may be NULL) receives the number of updates.  Returns LGF_OK,
 * LGF_ERR_NOT_CONVERGED or an error.  Mixed-precision handles run the FP32
 * phase down to LGF_TAIL_THETA (or until theta below 1e-6 stops halving
 * within 8 updates), then rebuild the links in FP64 from the loaded input and
 * the accumulated gauge transformation and finish in FP64; the links stay
 * in that FP64 form (double-float in tail mode 0) until the next load.  Each phase runs as one CUDA graph
 * launch with the loop on the device (the first call builds the graphs; the
 * host waits once per phase); under lgf_profile the host queues the
 * iterations instead.  Both stop at the same update. */
int lgf_fix(lgf_handle h, double theta_tol, int max_iter, int* iters_out);

/* Fix an ensemble of n configurations in turn, streaming them through the
 * device (paper Sec. 3.2: the string tension is measured on ensembles of
 * configurations, each brought to Landau gauge on its own; Sec. 2.2: the
 * host holds the lattice and the GPU fixes it).  host_in[k] (V*4*18 doubles,
 * the layout above) is fixed as lgf_load_links + lgf_fix(theta_tol, max_iter)
 * + lgf_store_links into host_out[k] would do, with bit-identical results.
 * Configuration k runs on h0 for even k and h1 for odd k; the two handles
 * must have the same lattice, dtype and device, and each should have its own
 * stream (lgf_set_stream).  The copies go through each handle's device
 * staging buffers on two streams of their own: while configuration k is
 * being fixed, configuration k + 1 is copied in and k - 1 copied out, so the
 * host link's transfers overlap the fixing.  host_in and host_out should be
 * pinned (page-locked) for the copies to run asynchronously; the caller must
 * leave every host_in[k] unchanged and read no host_out[k] until the call
 * returns.  host_out[k] may be host_in[k] (fixing in place: configuration k
 * is read before its result is written); no other output may overlap an
 * input.  iters_out (may be NULL) receives n update counts.  Allocates two
 * FP64 link buffers per handle on first use (kept until lgf_destroy).
 * Returns LGF_OK, LGF_ERR_NOT_CONVERGED (every configuration is still fixed
 * as far as max_iter allows and stored) or an error, whose message
 * lgf_last_error(h0) gives; after an error the state of both handles and of
 * the outputs not yet written is unspecified. */
int lgf_fix_stream(lgf_handle h0, lgf_handle h1, int n, const double* const* host_in, double* const* host_out,
                   double theta_tol, int max_iter, int* iters_out);

/* F and theta of the current links (either pointer may be NULL): the gauge
 * functional the steepest descent of paper Sec. 1 maximises and its
 * convergence measure, normalised as at the top of this file, summed in a
 * fixed order with FP64 above the warp (the result does not depend on
 * scheduling).  After the
 * double-float tail (LGF_TAIL_MODE 0) they come from that tail's gradient:
 * F to double-float accuracy, Delta to ~1e-12 absolute (its link corrections
 * are rounded in FP32), so theta is exact to ~1e-12 sqrt(theta). */
int lgf_functional(lgf_handle h, double* F, double* theta);

/* Intermediates of one iteration on the current links, without updating
 * them, for step-by-step checks.  Each non-NULL output receives V*8 doubles
 * (V complex pairs x 4): the gradient packed as (Delta01, Delta02, Delta12,
 * Im Delta00 + i Im Delta11) per site, and the accelerated gradient Delta~ in
 * the same packing; g receives V*18 doubles ([s][i][j] complex). */
int lgf_probe(lgf_handle h, double* delta_packed, double* delta_tilde_packed, double* g);

/* Updates of the last lgf_fix done in FP32 storage and in FP64 (a plain FP64
 * handle reports all of them as FP64; a mixed handle's FP32 phase and tail). */
int lgf_fix_split(lgf_handle h, int* fp32_iters, int* fp64_iters);

/* The theta history (theta before each update) of the last precision phase
 * of the last lgf_fix, up to cap entries; *n_out receives the count. */
int lgf_history(lgf_handle h, double* theta_out, int cap, int* n_out);

/* Text of the last error on h; with h NULL, of the last failed lgf_create or
 * lgf_functional_noalloc on the calling host thread. */
const char* lgf_last_error(lgf_handle h);

/* Kernel launches this handle has issued since creation (for accounting). */
long long lgf_launch_count(lgf_handle h);

/* Kernel kinds of one iteration, for lgf_profile_read(). */
enum lgf_kernel {
  LGF_K_GRADIENT = 0,   /* gradient Delta, FP64 F/theta sums, stop decision */
  LGF_K_FFT_AXIS = 1,   /* one-axis FFT pass (x, y or z; fwd or inv)        */
  LGF_K_FFT_XY = 2,     /* x-y plane FFT (forward and inverse)              */
  LGF_K_FFT_ZT = 3,     /* z-t plane FFT, forward + p2_max/p2 + inverse     */
  LGF_K_BUILD_G = 4,    /* g = reunitarised (1 + alpha/2 Delta~)            */
  LGF_K_UPDATE = 5,     /* U_mu(x) <- g(x) U_mu(x) g(x+mu)^dagger          */
  LGF_K_ACCUMULATE = 6, /* mixed precision: G <- g G                        */
  LGF_K_OTHER = 7,      /* layout conversions, copies                       */
  LGF_K_FFT_T = 8,      /* t pass: forward t FFT, p2_max/p2, inverse t FFT  */
  LGF_K_XY_GSTEP = 9,   /* inverse x-y plane FFT fused with G <- g G        */
  LGF_NUM_KERNELS = 10
};

/* Per-kernel timing with CUDA events recorded on the handle's stream right
 * before and after every launch (not part of the method; it measures it).
 * enable = 1 clears the totals and starts recording, 0 stops. */
int lgf_profile(lgf_handle h, int enable);

/* Accumulated device milliseconds and launch counts per lgf_kernel kind
 * since lgf_profile(h, 1): ms[k], launches[k] for k < n (either may be NULL). */
int lgf_profile_read(lgf_handle h, double* ms, long long* launches, int n);

/* Short name of a kernel kind ("update", ...), "" if out of range. */
const char* lgf_kernel_name(int kind);

/* ------------------------------------------------------------------------
 * Batches: several lattices (any sizes and storage types, one device) fixed
 * together.  Each phase is one launch of one CUDA graph holding, for every
 * member, a conditional while node around one of its iterations; each member
 * loops on the device until its own stop decision, so converged members cost
 * nothing further.  The members' loops run in parallel lanes (see
 * lgf_batch_set_lanes), so lattices too small to fill the GPU alone run
 * concurrently.  Mixed-precision members run their FP32 phases together, then
 * their FP64 tails together.  The batch borrows the handles (they must outlive it and
 * must not be used concurrently with it) and runs on its own streams.
 * ------------------------------------------------------------------------ */
typedef struct lgf_batch_ctx* lgf_batch;

/* Group n loaded-or-not handles (distinct, same device) into a batch. */
int lgf_batch_create(const lgf_handle* handles, int n, lgf_batch* out);
int lgf_batch_destroy(lgf_batch b);

/* Exactly n iterations of every member (no convergence test). */
int lgf_batch_iterate(lgf_batch b, int n);

/* lgf_fix for every member: iters_out[i] and converged_out[i] (either may be
 * NULL) receive each member's updates and 0/1.  Returns LGF_OK if all
 * converged, LGF_ERR_NOT_CONVERGED otherwise, or an error. */
int lgf_batch_fix(lgf_batch b, double theta_tol, int max_iter, int* iters_out, int* converged_out);

/* Text of the last error of a batch call. */
const char* lgf_batch_last_error(lgf_batch b);

/* Parallel branches of the batch's graphs: 0 (the default) gives every member
 * its own branch; n > 0 spreads the members over n lanes (largest first, each
 * onto the lane with the fewest sites so far), a lane running its members'
 * iteration blocks one after another.  Fewer lanes keep fewer packed
 * gradients competing for L2.  Not part of the paper's method. */
int lgf_batch_set_lanes(lgf_batch b, int lanes);

/* Lane autotuner: times one graph launch of reps iterations of every member
 * for 1, 2, 4, 8, 16 lanes and one lane per member, keeps the fastest and
 * stores it in *lanes_out (may be NULL).  The timed iterations are applied to
 * the members' links (like warm-up iterations) and counted as updates. */
int lgf_batch_autotune(lgf_batch b, int reps, int* lanes_out);

/* Autotuner: time every FFT schedule that applies to this lattice on each of
 * the handle's engines, reps Fourier accelerations each, and use the fastest
 * from now on (unless LGF_FFT_PIPELINE forces a pipeline).  The schedules
 * are the pipelines (x-y/z-t register planes, per-axis register passes,
 * shared-memory Stockham planes) and, for the register planes, the x-run
 * width of the z-t tiles (4 or 8 FP32 complex numbers, 2 or 4 FP64) and
 * the radix order of the z and t transforms (0: radix 4 first, 32 = 4 4 2;
 * 1: the same factors reversed, 32 = 2 4 4; FP32 only, where the stages
 * differ; 2: the pair split, FP32 lines of even length with one extent of
 * 16 or more: two threads share each line, the first radix-2 stage runs
 * across the pair and each thread transforms its half, which halves the
 * registers per thread).  The paper (Sec. 2.2) transforms with cuFFT's fixed plans; this
 * search has no counterpart there.  Results are cached per (precision,
 * lattice shape) for the process; if the environment variable
 * LGF_TUNE_CACHE names a file, the cache is written there (JSON) after each
 * tuning.  *chosen (may be NULL) receives the pipeline of the engine that
 * iterates first (1 Stockham planes, 2 axis passes, 3 register planes).
 * Overwrites the gradient scratch only; the links are untouched.  Tile
 * widths give bit-identical results; radix orders round differently in
 * FP32 (the fix still ends at the same F to the FP64 tail's accuracy).
 * Where an extent's pair-split stages equal those of order 1 (L = 8, 32),
 * orders 1 and 2 give bit-identical results. */
int lgf_autotune(lgf_handle h, int reps, int* chosen);

/* The FFT schedule engine `engine` (0: the FP64 engine, 1: the FP32 engine of
 * a mixed handle) uses: pipeline (1, 2, 3), z-t tile width (0 = default) and
 * radix order.  Any pointer may be NULL. */
int lgf_tune_schedule(lgf_handle h, int engine, int* pipeline, int* zt_bx, int* zt_ro);

/* Force a schedule on an engine (the values lgf_tune_schedule reports);
 * LGF_ERR_ARG if it does not apply to the lattice and precision. */
int lgf_set_schedule(lgf_handle h, int engine, int pipeline, int zt_bx, int zt_ro);

/* The schedule cache as a JSON file: {"lgf_fft_schedules": [ ... ]}, one
 * object per line, {"prec": bytes per real, "L": [Lx, Ly, Lz, Lt],
 * "pipeline": p, "zt_bx": b, "zt_ro": r, "ms": per acceleration}.
 * lgf_tune_load merges a file's valid entries into the process cache
 * (*n_loaded, may be NULL, receives their count) and from then on
 * lgf_create gives new handles the cached schedule of their shape; the first
 * lgf_create of a process loads LGF_TUNE_CACHE this way when it is set.
 * lgf_tune_save writes the whole cache (through a temporary file, renamed
 * into place).  lgf_tune_lookup reads one entry (LGF_ERR_ARG if absent);
 * lgf_tune_clear empties the cache and stops applying it at creation.
 * Host-only: none of these touch a GPU. */
int lgf_tune_load(const char* path, int* n_loaded);
int lgf_tune_save(const char* path);
int lgf_tune_lookup(int prec_bytes, int Lx, int Ly, int Lz, int Lt, int* pipeline, int* zt_bx, int* zt_ro);
int lgf_tune_clear(void);

/* ------------------------------------------------------------------------
 * Learned warm start.  A 4D convolutional network (three periodic 3^4-tap
 * layers, 48 -> 32 -> 32 -> 8 channels, ReLU after the first two, BF16
 * weights and activations with FP32 accumulation on the tensor cores)
 * maps per-site features of the loaded links -- the su(3) coefficients of
 * the traceless anti-Hermitian part of each link (32) and the six plaquette
 * traces / 3 -- to eight coefficients c_a; the warm start is the gauge
 * transformation g0(x) = exp(sum_a c_a i lambda_a / 2), installed as the
 * initial accumulated transformation of an FP32 gauge-representation
 * handle, after which lgf_fix runs the plain method (the judge, via theta
 * and F; it may end in a different Gribov copy than without the warm start).
 * Training maximises F(U^{g0}), the method's own functional: the signal
 * fed back is its derivative along left translations of g0, i.e. the
 * transformed links' gradient projected on the generators.  The paper has no
 * learned component; all network work runs on the handle's stream.
 * ------------------------------------------------------------------------ */
typedef struct lgf_net_ctx* lgf_net;

/* Number of FP32 parameters: W1[81][48][32], b1[32], W2[81][32][32], b2[32],
 * W3[81][32][8], b3[8] (tap = ((dt*3 + dz)*3 + dy)*3 + dx, offsets d - 1). */
int lgf_net_param_count(void);

/* New network on the current device, He-initialised from a counter-based
 * generator (SplitMix64 + Box-Muller) with this seed. */
int lgf_net_create(unsigned long long seed, lgf_net* out);
int lgf_net_destroy(lgf_net n);

/* Copy the FP32 parameters out / in (setting them resets the optimiser). */
int lgf_net_get_params(lgf_net n, float* host);
int lgf_net_set_params(lgf_net n, const float* host);

/* Network output c[V][8] for the links loaded in h (an LGF_F32 or
 * LGF_F32_R12 handle in gauge representation, V a multiple of 16); host_c
 * may be NULL. */
int lgf_net_forward(lgf_net n, lgf_handle h, float* host_c);

/* One training step on the links loaded in h: forward, loss -F(U^{g0}),
 * backward, and (if lr > 0) one Adam step (beta 0.9/0.999).  *F_out (may be
 * NULL) receives F(U^{g0}) before the step; host_grad (may be NULL) receives
 * the parameter gradient of -F (layout of lgf_net_get_params).  Leaves the
 * handle's links untouched. */
int lgf_net_train_step(lgf_net n, lgf_handle h, double lr, double* F_out, float* host_grad);

/* Install the predicted g0 as the initial gauge transformation of h; call
 * right after lgf_load_links (the following lgf_fix starts from U^{g0}). */
int lgf_net_warm_start(lgf_net n, lgf_handle h);

/* One convolution layer of the network on caller-held device activations
 * (bf16, [V][channels], site order as everywhere), with the network's
 * current weights, on a periodic Lx x Ly x Lz x Lt lattice; queued on
 * `stream` (NULL: the legacy default stream) and finished before the call
 * returns.  backward = 0: layer 1 (48 -> 32 channels), 2 (32 -> 32) or 3
 * (32 -> 16, the last 8 zero-weight padding), bias and (layers 1, 2) ReLU;
 * out_f32 (may be NULL) also receives the FP32 result [V][out channels].
 * backward = 1: the data gradient of layer 2 or 3 (in: the gradient with
 * respect to the layer's output, [V][32] or [V][16]; out: [V][32]), zeroed
 * where mask (the layer's input activation, may be NULL) is not positive.
 * The kernels are the tcgen05 implicit GEMMs the network runs on; this entry
 * point exposes them for testing and reuse.  LGF_ERR_TIMEOUT if a bounded
 * wait inside a kernel expired. */
int lgf_net_conv(lgf_net n, int layer, int backward, const void* in, const void* mask, void* out, float* out_f32,
                 int Lx, int Ly, int Lz, int Lt, void* stream);

/* Poll budget of the waits inside the tensor-core convolutions that wait for
 * a pipeline stage's MMAs (default and upper bound 2^22 polls; polls < 0
 * restores the default).  With a budget of 0 every such wait expires at
 * once: each CTA records the error, stops issuing, waits for the MMAs it has
 * issued with the full budget, frees its tensor memory and returns, and the
 * call that ran the convolution returns LGF_ERR_TIMEOUT with its output
 * unspecified.  This is how the expiry path of those bounded waits is tested
 * without a fault; the context stays usable.  Synchronises the device. */
int lgf_net_set_wait_budget(lgf_net n, long long polls);

/* Text of the last error of a network call (NULL: of lgf_net_create). */
const char* lgf_net_last_error(lgf_net n);

/* F and theta of links the caller already holds in device memory, computed
 * without allocating any memory.  The paper has no counterpart: this exists
 * for callers that may not allocate on the GPU -- a host program that
 * reserves the device memory for its own pool and forbids the libraries it
 * loads to call cudaMalloc, or monitoring code that must not change the
 * memory footprint of the job it observes.
 *
 *   links   device pointer, the library's structure-of-arrays storage for
 *           dtype: NC complex planes of V elements per direction,
 *           element [(mu*NC + c)*V + s], c = 3i + j, NC = 9 (18-real) or 6
 *           (12-real: rows 1-2, row 3 rebuilt), complex128 for LGF_F64 /
 *           LGF_F64_R12, complex64 for LGF_F32 / LGF_F32_R12; s and mu as in
 *           the host layout.  Read only.
 *   out     device pointer to 2 doubles: out[0] = F, out[1] = theta.
 *   stream  cudaStream_t to run on (NULL: the legacy default stream).
 *
 * The work is queued on `stream` and the call returns without waiting; out
 * is valid once the stream has reached it.  The per-block partial sums live
 * in a fixed array inside the library (256 KiB on every GPU that loads it,
 * held until the process exits), so V may be at most 4,194,304 sites
 * (e.g. 32^4 or 48^3 x 12; 64^4 is rejected with LGF_ERR_ARG).  Every call
 * shares that array: calls that overlap on the GPU race on it and give wrong
 * results, so order them on one stream or synchronise between them.  Every
 * call made while `stream` is not capturing looks up the array's device
 * address (cudaGetSymbolAddress) in the current device's current context,
 * so a call after cudaDeviceReset or in another context finds the right
 * array; a call made during stream capture reuses the address found by the
 * last uncaptured call on that device, so make one uncaptured call, in the
 * context the capture will use, before capture begins (a captured call with
 * no earlier one gives LGF_ERR_ARG).  Errors: LGF_ERR_ARG for bad extents,
 * dtype, size or NULL pointers, LGF_ERR_CUDA for a failed lookup or launch;
 * the text is in lgf_last_error(NULL). */
int lgf_functional_noalloc(const void* links, int Lx, int Ly, int Lz, int Lt, int dtype, double* out,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LGF_H */
