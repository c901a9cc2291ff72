// oci_device.cuh -- device helpers shared by the sweep kernels: the stop rule of
// Sec. 2.1 applied to the device state, and the "last block finishes" pattern
// that lets a sweep kernel end with its own norm reduction (no separate
// finalize launch per sweep).
#pragma once
#include <math.h>

#include "oci_internal.h"

namespace oci {

// Fixed-order sum of p[0:n) by the whole block; the result is valid in thread 0.
// Loads bypass L1 (the partials were written by other blocks of this launch).
__device__ __forceinline__ double block_sum_fixed(const double *p, int n, double *red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  double s = 0.0;
  for (int i = tid; i < n; i += nthr) s += __ldcg(p + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();  // red may still be read by the caller's previous reduction
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (tid == 0)
    for (int w = 0; w < (nthr + 31) / 32; w++) t += red[w];
  return t;
}

// Publish this block's partial; returns true (in every thread) in the block that
// finished last.  That block resets the counter for the next launch.
__device__ __forceinline__ bool publish_partial(double *partials, int slot, double v, unsigned *counter,
                                                unsigned nblocks, bool *flag) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) {
    partials[slot] = v;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    *flag = prev == nblocks - 1;
  }
  __syncthreads();
  const bool last = *flag;
  if (last) __threadfence();
  return last;
}

// Grid barrier on a 64-bit arrival count that only grows within a launch (the
// host zeroes it before the launch); thread 0 of every block.  Episode k of
// the launch (k = 1, 2, ...) is passed once the count reaches k * nblocks: one
// atomic add with acquire-release semantics per block (release publishes the
// block's writes, ordered before it by the caller's __syncthreads; acquire
// makes the last block to arrive see everyone else's) and acquire loads while
// waiting -- no separate fences, no reset by the last block.  The spin is
// bounded by `limit`; false when it gave up.
__device__ __forceinline__ bool grid_barrier_count(unsigned long long *count, unsigned long long target,
                                                   long long limit) {
  unsigned long long v;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(v) : "l"(count) : "memory");
  if (v + 1 >= target) return true;
  for (long long k = 0; k < limit; k++) {
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(count) : "memory");
    if (v >= target) return true;
    __nanosleep(32);
  }
  return false;
}

// Stop rule of Sec. 2.1 (Algorithm 2) for the FP64 forms; one thread.
__device__ __forceinline__ void finish_fp64(DevState *ds, double *e_hist, double e, cudaGraphConditionalHandle cond,
                                            int use_cond) {
  DevState d = *ds;  // one load of the state, one store below
  const int l = d.l;
  if (e_hist && l < d.max_iter) e_hist[l] = e;
  double rho = 0.0;
  int conv = 0;
  if (!isfinite(e)) {
    d.status = OCI_E_NONFINITE;
    d.done = 1;
  } else {
    if (l >= 1 && d.e_prev > 0.0) rho = e / d.e_prev;
    if (!d.fixed) {
      if (e == 0.0) conv = 1;
      else if (l >= 1) conv = e < d.tol * (1.0 - rho);
    }
  }
  d.e = e;
  d.rho = rho;
  d.e_prev = e;
  d.l = l + 1;
  if (!d.inplace) d.cur ^= 1;
  if (!d.fixed && !d.done) {
    if (conv) {
      d.status = OCI_OK;
      d.done = 1;
    } else if (l + 1 >= d.max_iter) {
      d.status = OCI_E_NOCONV;
      d.done = 1;
    }
  }
  *ds = d;
  if (use_cond && d.done) cudaGraphSetConditional(cond, 0);
}

// Stop rule and refinement decision of the mixed-precision forms; one thread.
// The stop rule is accepted only where the low-precision correction is small:
// on the first sweep after a refinement (delta = A~^{-1} r from a fresh FP64
// residual) or in a block that began below tol.  Otherwise refine first and test
// the next sweep again.
__device__ __forceinline__ void finish_mixed(DevState *ds, double *e_hist, double e, cudaGraphConditionalHandle cond,
                                             int use_cond) {
  DevState d = *ds;
  if (d.refine) {  // settle the refinement made by the previous body's outer kernel
    d.cur ^= 1;
    d.refine = 0;
    d.blk_i = 0;
  }
  const int l = d.l;
  if (e_hist && l < d.max_iter) e_hist[l] = e;
  double rho = 0.0;
  int conv = 0;
  if (!isfinite(e)) {
    d.status = OCI_E_NONFINITE;
    d.done = 1;
  } else {
    if (l >= 1 && d.e_prev > 0.0) rho = e / d.e_prev;
    if (!d.fixed) {
      if (e == 0.0) conv = 1;
      else if (l >= 1) conv = e < d.tol * (1.0 - rho);
    }
  }
  d.e = e;
  d.rho = rho;
  d.e_prev = e;
  d.l = l + 1;
  if (!d.inplace) d.dcur ^= 1;  // red-black: one correction buffer updated in place
  d.blk_i += 1;
  if (d.blk_i == 1) d.e_blk0 = e;
  int verify = 0;
  if (conv && !(d.blk_i == 1 || d.e_blk0 <= d.tol)) {
    conv = 0;
    verify = 1;
  }
  if (!d.fixed && !d.done) {
    if (conv) {
      d.status = OCI_OK;
      d.done = 1;
    } else if (l + 1 >= d.max_iter) {
      d.status = OCI_E_NOCONV;
      d.done = 1;
    }
  }
  const int refine = d.done || verify || d.blk_i >= d.k_max || e < d.theta * d.e_blk0;
  d.refine = refine;
  if (refine) d.n_refine += 1;
  *ds = d;
  if (use_cond && d.done) cudaGraphSetConditional(cond, 0);
  // in the graph the refinement kernel runs under an IF node (no handle: always launched)
  if (use_cond && d.cond_ref) cudaGraphSetConditional((cudaGraphConditionalHandle)d.cond_ref, refine);
}

}  // namespace oci
