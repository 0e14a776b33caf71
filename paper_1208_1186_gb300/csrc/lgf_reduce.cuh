// Block and grid reductions of (Re Tr U, Tr Delta Delta^dagger) and the stop
// decision of an iteration queue, shared by the gradient kernels.
//
// Per-site terms and the sum over a warp are taken in the storage precision T;
// everything above the warp (warps of a block, blocks of the grid) is summed
// in FP64, in a fixed order, so that the result does not depend on which
// block finishes last.  (With T = double every stage is FP64.)  On GB300 the
// FP64 pipe runs at about 1/60 of the FP32 rate, so keeping the per-site and
// per-warp stages in FP32 for FP32 storage is what keeps the gradient kernel
// memory-bound.
#pragma once

#include "lgf_common.cuh"

namespace lgf {

// Sum per-warp totals over the block in FP64, in warp order; the totals are
// read from lane 0 of each warp and the result is valid in thread 0.
__device__ __forceinline__ void block_sum_warp_totals(double wa, double wb, double& ra, double& rb) {
  __shared__ double sa[32], sb[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = wa;
    sb[w] = wb;
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double x = 0.0, y = 0.0;
  if (w == 0) {
    x = l < nw ? sa[l] : 0.0;
    y = l < nw ? sb[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
  }
  ra = x;
  rb = y;
}

// Sum (a, b) over the block; the result is valid in thread 0.
template <class T>
__device__ __forceinline__ void block_sum_mixed(T a, T b, double& ra, double& rb) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  block_sum_warp_totals((double)a, (double)b, ra, rb);
}

// F, theta and the stop decision from the grid sums (one thread).
__device__ __forceinline__ void finish_reduction(DevState* st, double fs, double ts, double normF, double normT,
                                                 int mode) {
  const double F = fs * normF, th = ts * normT;
  st->F = F;
  st->theta = th;
  const bool bad = !isfinite(F) || !isfinite(th);
  if (bad) st->nonfinite = 1;
  if (mode != 1) return;
  if (st->hist != nullptr && st->iters < st->hist_cap) st->hist[st->iters] = th;
  bool stop = bad || (st->tol >= 0.0 && th < st->tol) || st->iters >= st->max_iter;
  if (!stop && st->stall && th < 1e-6) {
    // the FP32 phase hands over once theta has not halved within 8 updates
    if (st->stall_ref > 0.0 && th > 0.5 * st->stall_ref && st->iters - st->stall_iters >= 8) {
      stop = true;
    } else if (st->stall_ref == 0.0 || th <= 0.5 * st->stall_ref) {
      st->stall_ref = th;
      st->stall_iters = st->iters;
    }
  }
  if (stop) {
    st->done = 1;
  } else {
    st->iters += 1;
  }
  if (st->use_cond) cudaGraphSetConditional(st->cond, stop ? 0u : 1u);
}

// Gradient kernels of an iteration queue: true if the queue has stopped, so
// the launch does nothing; in a device-side graph loop the first thread of
// the grid also ends the loop (one caller of cudaGraphSetConditional).
__device__ __forceinline__ bool queue_stopped(const DevState* st, int mode) {
  if (mode != 1 || !st->done) return false;
  if (st->use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(st->cond, 0u);
  return true;
}

// Block sums (valid in thread 0) -> grid result: every block stores its pair;
// the last block to arrive adds all pairs in index order and finishes the
// reduction.  Must be called by every thread of every block.
__device__ __forceinline__ void grid_reduce_block_sums(double a, double b, double2* __restrict__ partial,
                                                       DevState* st, double normF, double normT, int mode) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = make_double2(a, b);
    __threadfence();
    const unsigned prev = atomicAdd(&st->arrive, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    const double2 p = __ldcg(partial + i);
    x += p.x;
    y += p.y;
  }
  __syncthreads();  // the shared scratch of the block sum is reused
  block_sum_mixed<double>(x, y, a, b);
  if (threadIdx.x == 0) {
    st->arrive = 0;
    finish_reduction(st, a, b, normF, normT, mode);
  }
}

// Per-thread terms -> grid result (warp sums in T, FP64 above the warp).
template <class T>
__device__ __forceinline__ void grid_reduce(T fs, T ts, double2* __restrict__ partial, DevState* st, double normF,
                                            double normT, int mode) {
  double a, b;
  block_sum_mixed<T>(fs, ts, a, b);
  grid_reduce_block_sums(a, b, partial, st, normF, normT, mode);
}

// Per-warp totals (valid in lane 0) -> grid result.
__device__ __forceinline__ void grid_reduce_warp_totals(double wf, double wt, double2* __restrict__ partial,
                                                        DevState* st, double normF, double normT, int mode) {
  double a, b;
  block_sum_warp_totals(wf, wt, a, b);
  grid_reduce_block_sums(a, b, partial, st, normF, normT, mode);
}

}  // namespace lgf
