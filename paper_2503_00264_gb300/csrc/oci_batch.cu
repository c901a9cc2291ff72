// oci_batch.cu -- batched form: many independent slabs of uneven size, angle
// order and group count advanced by one graph launch per time step.
//
// Slabs are grouped by (N, G) into classes.  Within a class the slabs are
// concatenated into one structure-of-arrays cell range ([G][N][4][Jc], cells
// fastest), each slab padded to a multiple of 128 cells so that no tile of the
// sweep and no 32-cell block of the carry straddles two slabs.  Per cell: the
// class-wide cell-type id (the type tables carry each slab's dt and speeds) and
// the slab index (-1 for padding).  Per slab: first cell, length, first and last
// tile, its own convergence state (DevState) and incident fluxes.
//
// The sweep kernel is persistent: a grid sized to the resident capacity loops
// over the class's tiles, skipping tiles of slabs that have converged.  The
// per-slab finalize (one warp per slab) applies the stop rule of Sec. 2.1 to
// that slab's norm; a device counter of unconverged slabs ends the conditional
// WHILE graph when it reaches zero.  The cell solve is the FP64 structured solve
// of oci_sweep.cu; the slab boundaries replace the inflow of the neighbouring
// cell by the slab's incident flux.
#include <math.h>

#include <algorithm>

#include "oci_batch.h"
#include "oci_cvt.cuh"
#include "oci_device.cuh"

namespace oci {

__global__ void k_b_step_const(int Jc, int N, int G, const int32_t *__restrict__ type,
                               const int32_t *__restrict__ seg, const double *__restrict__ tdx,
                               const double *__restrict__ tah, const double *__restrict__ Q,
                               const double *__restrict__ psi_prev, const double *__restrict__ Linv,
                               double *__restrict__ tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int gm = blockIdx.y;
  if (j >= Jc || seg[j] < 0) return;
  const int g = gm / N;
  const int tau = type[j];
  const double dx = tdx[tau];
  const double ah = tah[(size_t)tau * G + g];
  double q[4] = {0.0, 0.0, 0.0, 0.0};
  if (Q) {
#pragma unroll
    for (int p = 0; p < 4; p++) q[p] = dx / 4.0 * Q[(size_t)(g * 4 + p) * Jc + j];
  }
  const double c0 = q[0] + ah * psi_prev[(size_t)(gm * 2 + 0) * Jc + j];
  const double c1 = q[1] + ah * psi_prev[(size_t)(gm * 2 + 1) * Jc + j];
  const double *L = Linv + ((size_t)tau * G * N + gm) * 16;
#pragma unroll
  for (int p = 0; p < 4; p++)
    tc[(size_t)(gm * 4 + p) * Jc + j] = L[p * 4 + 0] * c0 + L[p * 4 + 1] * c1 + L[p * 4 + 2] * q[2] + L[p * 4 + 3] * q[3];
}

// Persistent batched sweep.  Block = CB cells x G groups; tiles of CB cells.
__global__ void __launch_bounds__(256) k_b_sweep(BatchClassDev c, DevState *__restrict__ ds) {
  extern __shared__ double sm[];
  const int CB = blockDim.x, N = c.N, G = c.G, Jc = c.Jc;
  const int cl = threadIdx.x, g = threadIdx.y;
  double *t_s = sm;
  double *y_s = sm + (size_t)G * N * 4 * CB;
  __shared__ double red[8];
  const int N2 = N / 2;
  // Tiles are dealt round-robin (tile t to block t mod grid); walk the slabs and
  // jump straight to this block's tiles of every slab that has not converged,
  // so converged slabs cost one flag read instead of one per tile.
  for (int s = 0; s < c.n_slabs; s++) {
    if (ds[s].done) continue;  // uniform over the block
    const int t0 = c.slab_tile0[s], t1 = c.slab_tile1[s];
    const int G_ = gridDim.x;
    const int first = t0 + (((int)blockIdx.x - t0 % G_) % G_ + G_) % G_;
    for (int tile = first; tile < t1; tile += G_) {
      const int cur = ds[s].cur;
      const double *__restrict__ Pin = cur ? c.Psi1 : c.Psi0;
      double *__restrict__ Pout = cur ? c.Psi0 : c.Psi1;
      const int j = c.tile_first_cell[tile] + cl;
      const int jl = j - c.slab_start[s];
      const int Js = c.slab_J[s];
      const bool active = jl < Js;
      const int tau = active ? c.type[j] : 0;
      const size_t tb = (size_t)tau * G * N;
      const double *inc = c.inc + (size_t)s * 2 * G * N * 2;
      double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
      if (active) {
  #pragma unroll 2
        for (int m = 0; m < N; m++) {
          const int gm = g * N + m;
          const size_t base = (size_t)gm * 4 * Jc + j;
          double uk, uh;
          if (m >= N2) {
            if (jl > 0) {
              uk = Pin[base + (size_t)Jc - 1];
              uh = Pin[base + 3 * (size_t)Jc - 1];
            } else {
              uk = inc[gm * 2 + 0];
              uh = inc[gm * 2 + 1];
            }
          } else {
            if (jl < Js - 1) {
              uk = Pin[base + 1];
              uh = Pin[base + 2 * (size_t)Jc + 1];
            } else {
              uk = inc[(G * N + gm) * 2 + 0];
              uh = inc[(G * N + gm) * 2 + 1];
            }
          }
          const double *C = c.Cin + (tb + gm) * 8;
          const double t0 = fma(C[1], uh, fma(C[0], uk, c.tc[base]));
          const double t1 = fma(C[3], uh, fma(C[2], uk, c.tc[base + (size_t)Jc]));
          const double t2 = fma(C[5], uh, fma(C[4], uk, c.tc[base + 2 * (size_t)Jc]));
          const double t3 = fma(C[7], uh, fma(C[6], uk, c.tc[base + 3 * (size_t)Jc]));
          double *ts = t_s + (size_t)(gm * 4) * CB + cl;
          ts[0] = t0;
          ts[CB] = t1;
          ts[2 * CB] = t2;
          ts[3 * CB] = t3;
          const double wm = c.w[m];
          y0 = fma(wm, t0, y0);
          y1 = fma(wm, t1, y1);
          y2 = fma(wm, t2, y2);
          y3 = fma(wm, t3, y3);
        }
        double *ys = y_s + (size_t)(g * 4) * CB + cl;
        ys[0] = y0;
        ys[CB] = y1;
        ys[2 * CB] = y2;
        ys[3 * CB] = y3;
      }
      __syncthreads();
      double e2 = 0.0;
      if (active) {
        const int G4 = 4 * G;
        const double *M = c.Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int k = 0; k < G4; k++) {
          const double yk = y_s[(size_t)k * CB + cl];
          s0 = fma(M[k], yk, s0);
          s1 = fma(M[G4 + k], yk, s1);
          s2 = fma(M[2 * G4 + k], yk, s2);
          s3 = fma(M[3 * G4 + k], yk, s3);
        }
  #pragma unroll 2
        for (int m = 0; m < N; m++) {
          const int gm = g * N + m;
          const size_t base = (size_t)gm * 4 * Jc + j;
          const double *L = c.Linv + (tb + gm) * 16;
          const double *ts = t_s + (size_t)(gm * 4) * CB + cl;
          double o[4];
  #pragma unroll
          for (int p = 0; p < 4; p++)
            o[p] = fma(L[p * 4 + 3], s3, fma(L[p * 4 + 2], s2, fma(L[p * 4 + 1], s1, fma(L[p * 4 + 0], s0, ts[p * CB]))));
  #pragma unroll
          for (int p = 0; p < 4; p++) {
            const double d = o[p] - Pin[base + (size_t)p * Jc];
            e2 = fma(d, d, e2);
            Pout[base + (size_t)p * Jc] = o[p];
          }
        }
      }
      // fixed-order block sum
      const int tid = threadIdx.y * CB + threadIdx.x;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
      if ((tid & 31) == 0) red[tid >> 5] = e2;
      __syncthreads();
      if (tid == 0) {
        double v = 0.0;
        for (int i = 0; i < (CB * G + 31) / 32; i++) v += red[i];
        c.partials[tile] = v;
      }
      __syncthreads();  // t_s / y_s / red reused by the next tile
    }
  }
}

// One block per slab: fixed-order sum of the slab's tile partials, stop rule,
// ping-pong flip; the last slab to finish ends the WHILE loop.
constexpr int kBFinThreads = 128;
__global__ void __launch_bounds__(kBFinThreads) k_b_finalize(BatchClassDev c, DevState *__restrict__ ds, int *active,
                                                            int use_cond, cudaGraphConditionalHandle cond) {
  __shared__ double red[kBFinThreads / 32];
  const int s = blockIdx.x;
  DevState &d = ds[s];
  if (d.done) return;  // uniform: thread 0 writes the state only after the barriers below
  const int t0 = c.slab_tile0[s];
  const double v = block_sum_fixed(c.partials + t0, c.slab_tile1[s] - t0, red);
  if (threadIdx.x != 0) return;
  const double e = sqrt(v);
  const int l = d.l;
  double rho = 0.0;
  int conv = 0;
  if (!isfinite(e)) {
    d.status = OCI_E_NONFINITE;
    d.done = 1;
  } else {
    if (l >= 1 && d.e_prev > 0.0) rho = e / d.e_prev;
    if (e == 0.0) conv = 1;
    else if (l >= 1) conv = e < d.tol * (1.0 - rho);
  }
  d.e = e;
  d.rho = rho;
  d.e_prev = e;
  d.l = l + 1;
  d.cur ^= 1;
  if (!d.done) {
    if (conv) {
      d.status = OCI_OK;
      d.done = 1;
    } else if (l + 1 >= d.max_iter) {
      d.status = OCI_E_NOCONV;
      d.done = 1;
    }
  }
  if (d.done) {
    const int before = atomicSub(active, 1);
    if (before == 1 && use_cond) cudaGraphSetConditional(cond, 0);
  }
}

// Commit of converged slabs: phi, carry and per-block balance tallies (as k_carry).
__global__ void __launch_bounds__(32 * kMaxG) k_b_carry(BatchClassDev c, const DevState *__restrict__ ds) {
  __shared__ double ph_s[kMaxG * 4][32];
  const int N = c.N, G = c.G, Jc = c.Jc;
  const int cl = threadIdx.x, g = threadIdx.y;
  const int j = blockIdx.x * 32 + cl;
  const int s = c.seg[blockIdx.x * 32];  // blocks never straddle slabs
  if (s < 0 || ds[s].status != OCI_OK) return;  // uniform
  const double *__restrict__ P = ds[s].cur ? c.Psi1 : c.Psi0;
  const bool active = c.seg[j] >= 0;
  double ph[4] = {0, 0, 0, 0}, pp[2] = {0, 0};
  int tau = 0;
  if (active) {
    tau = c.type[j];
    for (int m = 0; m < N; m++) {
      const int gm = g * N + m;
      const double wm = c.w[m];
      const size_t base = (size_t)gm * 4 * Jc + j;
      double o[4];
#pragma unroll
      for (int p = 0; p < 4; p++) {
        o[p] = P[base + (size_t)p * Jc];
        ph[p] = fma(wm, o[p], ph[p]);
      }
      const size_t pb = (size_t)gm * 2 * Jc + j;
      pp[0] = fma(wm, c.psi_prev[pb], pp[0]);
      pp[1] = fma(wm, c.psi_prev[pb + Jc], pp[1]);
      c.psi_prev[pb] = o[2];
      c.psi_prev[pb + Jc] = o[3];
    }
#pragma unroll
    for (int p = 0; p < 4; p++) {
      c.phi[(size_t)(g * 4 + p) * Jc + j] = ph[p];
      ph_s[g * 4 + p][cl] = ph[p];
    }
  }
  __syncthreads();
  double tally[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (active) {
    const double dx = c.tdx[tau];
    const double sig = c.tsig[(size_t)tau * G + g];
    const double rate = 2.0 * c.tah[(size_t)tau * G + g];  // dx / (v dt)
    tally[0] = rate / 2.0 * ((ph[2] - pp[0]) + (ph[3] - pp[1]));
    tally[1] = rate * ((ph[2] - ph[0]) + (ph[3] - ph[1]));
    tally[2] = dx / 2.0 * sig * (ph[0] + ph[1]);
    tally[3] = dx / 2.0 * sig * (ph[2] + ph[3]);
    for (int gp = 0; gp < G; gp++) {
      const double k2 = 2.0 * c.Kap[((size_t)tau * G + gp) * G + g];
      tally[4] += k2 * (ph_s[gp * 4 + 0][cl] + ph_s[gp * 4 + 1][cl]);
      tally[5] += k2 * (ph_s[gp * 4 + 2][cl] + ph_s[gp * 4 + 3][cl]);
    }
    if (c.Q) {
      tally[6] = dx / 2.0 * (c.Q[(size_t)(g * 4 + 0) * Jc + j] + c.Q[(size_t)(g * 4 + 1) * Jc + j]);
      tally[7] = dx / 2.0 * (c.Q[(size_t)(g * 4 + 2) * Jc + j] + c.Q[(size_t)(g * 4 + 3) * Jc + j]);
    }
  }
#pragma unroll
  for (int k = 0; k < 8; k++) {
    double x = tally[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (cl == 0) c.bal_partials[((size_t)blockIdx.x * G + g) * 8 + k] = x;
  }
}

// Per (slab, group): fixed-order sum of the slab's carry blocks plus leakage.
__global__ void k_b_balance_final(BatchClassDev c, const DevState *__restrict__ ds) {
  const int s = blockIdx.x, g = blockIdx.y;
  if (threadIdx.x != 0 || ds[s].status != OCI_OK) return;
  const int N = c.N, G = c.G, Jc = c.Jc;
  const int b0 = c.slab_start[s] / 32, b1 = (c.slab_start[s] + c.slab_J[s] + 31) / 32;
  double tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = b0; b < b1; b++)
    for (int k = 0; k < 8; k++) tot[k] += c.bal_partials[((size_t)b * G + g) * 8 + k];
  const double *P = ds[s].cur ? c.Psi1 : c.Psi0;
  const double *inc = c.inc + (size_t)s * 2 * G * N * 2;
  const int jf = c.slab_start[s], jlast = c.slab_start[s] + c.slab_J[s] - 1;
  double lA = 0.0, lE = 0.0;
  for (int m = 0; m < N; m++) {
    const int gm = g * N + m;
    double rk, rh, lk, lh;
    if (c.mu[m] > 0) {
      rk = P[(size_t)(gm * 4 + 1) * Jc + jlast];
      rh = P[(size_t)(gm * 4 + 3) * Jc + jlast];
      lk = inc[gm * 2 + 0];
      lh = inc[gm * 2 + 1];
    } else {
      lk = P[(size_t)(gm * 4 + 0) * Jc + jf];
      lh = P[(size_t)(gm * 4 + 2) * Jc + jf];
      rk = inc[(G * N + gm) * 2 + 0];
      rh = inc[(G * N + gm) * 2 + 1];
    }
    lA += c.w[m] * c.mu[m] * (rk - lk);
    lE += c.w[m] * c.mu[m] * (rh - lh);
  }
  double *bg = c.bal + ((size_t)s * G + g) * 10;
  bg[0] = tot[0]; bg[1] = lA; bg[2] = tot[2]; bg[3] = tot[4]; bg[4] = tot[6];
  bg[5] = tot[1]; bg[6] = lE; bg[7] = tot[3]; bg[8] = tot[5]; bg[9] = tot[7];
}

// ---------------------------------------------------------------- mixed form
// The mixed-precision form of oci_mixed.cu per slab: every slab has its own
// FP32 correction state (ping-pong index, block count, refinement flag) in its
// DevState and the same stop rule / refinement decisions (finish_mixed).

// c = dx/4 Q + dx/(2 v dt) psi_prev on rows kL, kR (Eq. rhs_sg), not pre-multiplied.
__global__ void k_b_mx_step_const(BatchClassDev c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int gm = blockIdx.y;
  const int N = c.N, G = c.G, Jc = c.Jc;
  if (j >= Jc || c.seg[j] < 0) return;
  const int g = gm / N;
  const int tau = c.type[j];
  const double dx = c.tdx[tau];
  const double ah = c.tah[(size_t)tau * G + g];
#pragma unroll
  for (int p = 0; p < 4; p++) {
    double v = c.Q ? dx / 4.0 * c.Q[(size_t)(g * 4 + p) * Jc + j] : 0.0;
    if (p < 2) v += ah * c.psi_prev[(size_t)(gm * 2 + p) * Jc + j];
    c.cvec[(size_t)(gm * 4 + p) * Jc + j] = v;
  }
}

// FP32 inner sweep on the tiles of the slabs still iterating (layout of k_b_sweep).
__global__ void __launch_bounds__(256) k_b_mx_inner(BatchClassDev c, const DevState *__restrict__ ds) {
  extern __shared__ float smf[];
  __shared__ double red[8];
  const int CB = blockDim.x, N = c.N, G = c.G, Jc = c.Jc;
  const int cl = threadIdx.x, g = threadIdx.y;
  float *t_s = smf;
  float *y_s = smf + (size_t)G * N * 4 * CB;
  const int N2 = N / 2;
  for (int s = 0; s < c.n_slabs; s++) {
    if (ds[s].done) continue;  // uniform
    const bool zero = ds[s].refine || ds[s].blk_i == 0;
    const int dcur = ds[s].dcur;
    const float *__restrict__ Din = dcur ? c.D1 : c.D0;
    float *__restrict__ Dout = dcur ? c.D0 : c.D1;
    const int t0 = c.slab_tile0[s], t1 = c.slab_tile1[s];
    const int G_ = gridDim.x;
    const int first = t0 + (((int)blockIdx.x - t0 % G_) % G_ + G_) % G_;
    for (int tile = first; tile < t1; tile += G_) {
      const int j = c.tile_first_cell[tile] + cl;
      const int jl = j - c.slab_start[s];
      const int Js = c.slab_J[s];
      const bool active = jl < Js;
      const int tau = active ? c.type[j] : 0;
      const size_t tb = (size_t)tau * G * N;
      float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
      if (active) {
        for (int m = 0; m < N; m++) {
          const int gm = g * N + m;
          const size_t base = (size_t)gm * 4 * Jc + j;
          float uk = 0.f, uh = 0.f;
          if (!zero) {
            if (m >= N2) {
              if (jl > 0) {
                uk = Din[base + (size_t)Jc - 1];
                uh = Din[base + 3 * (size_t)Jc - 1];
              }
            } else if (jl < Js - 1) {
              uk = Din[base + 1];
              uh = Din[base + 2 * (size_t)Jc + 1];
            }
          }
          const float *C = c.Cin32 + (tb + gm) * 8;
          const float t0v = fmaf(C[1], uh, fmaf(C[0], uk, c.z32[base]));
          const float t1v = fmaf(C[3], uh, fmaf(C[2], uk, c.z32[base + (size_t)Jc]));
          const float t2v = fmaf(C[5], uh, fmaf(C[4], uk, c.z32[base + 2 * (size_t)Jc]));
          const float t3v = fmaf(C[7], uh, fmaf(C[6], uk, c.z32[base + 3 * (size_t)Jc]));
          float *ts = t_s + (size_t)(gm * 4) * CB + cl;
          ts[0] = t0v;
          ts[CB] = t1v;
          ts[2 * CB] = t2v;
          ts[3 * CB] = t3v;
          const float wm = c.w32[m];
          y0 = fmaf(wm, t0v, y0);
          y1 = fmaf(wm, t1v, y1);
          y2 = fmaf(wm, t2v, y2);
          y3 = fmaf(wm, t3v, y3);
        }
        float *ys = y_s + (size_t)(g * 4) * CB + cl;
        ys[0] = y0;
        ys[CB] = y1;
        ys[2 * CB] = y2;
        ys[3 * CB] = y3;
      }
      __syncthreads();
      float e2 = 0.f;
      if (active) {
        const int G4 = 4 * G;
        const float *M = c.Mp32 + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (int k = 0; k < G4; k++) {
          const float yk = y_s[(size_t)k * CB + cl];
          s0 = fmaf(M[k], yk, s0);
          s1 = fmaf(M[G4 + k], yk, s1);
          s2 = fmaf(M[2 * G4 + k], yk, s2);
          s3 = fmaf(M[3 * G4 + k], yk, s3);
        }
        for (int m = 0; m < N; m++) {
          const int gm = g * N + m;
          const size_t base = (size_t)gm * 4 * Jc + j;
          const float *L = c.Linv32 + (tb + gm) * 16;
          const float *ts = t_s + (size_t)(gm * 4) * CB + cl;
#pragma unroll
          for (int p = 0; p < 4; p++) {
            const float o = fmaf(L[p * 4 + 3], s3, fmaf(L[p * 4 + 2], s2, fmaf(L[p * 4 + 1], s1, fmaf(L[p * 4 + 0], s0, ts[p * CB]))));
            const float d = zero ? o : o - Din[base + (size_t)p * Jc];
            e2 = fmaf(d, d, e2);
            Dout[base + (size_t)p * Jc] = o;
          }
        }
      }
      double v = (double)e2;
      const int tid = threadIdx.y * CB + threadIdx.x;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double acc = 0.0;
        for (int i = 0; i < (CB * G + 31) / 32; i++) acc += red[i];
        c.partials[tile] = acc;
      }
      __syncthreads();
    }
  }
}

// One block per slab: fixed-order sum of its tile partials, then the mixed-form
// stop rule and refinement decision; the last slab to finish ends the loop.  In
// the graph the class's refinement kernel sits under an IF node: the last
// block of this launch (counter in flags[1]) sets it to whether any slab of the
// class asked for a refinement (flags[0]) and resets both words.
__global__ void __launch_bounds__(kBFinThreads) k_b_mx_finalize(BatchClassDev c, DevState *__restrict__ ds,
                                                               int *active, int use_cond,
                                                               cudaGraphConditionalHandle cond,
                                                               unsigned *flags, cudaGraphConditionalHandle if_cond) {
  __shared__ double red[kBFinThreads / 32];
  const int s = blockIdx.x;
  int refine = 0;
  if (ds[s].done) {
    // a slab that finished in the previous body: its last refinement has been
    // applied by that body's outer kernel; settle it so no later body repeats it
    if (threadIdx.x == 0 && ds[s].refine) {
      ds[s].cur ^= 1;
      ds[s].refine = 0;
      ds[s].blk_i = 0;
    }
  } else {
    const int t0 = c.slab_tile0[s];
    const double v = block_sum_fixed(c.partials + t0, c.slab_tile1[s] - t0, red);
    if (threadIdx.x == 0) {
      finish_mixed(&ds[s], nullptr, sqrt(v), cond, 0);
      refine = ds[s].refine;
      if (ds[s].done) {
        const int before = atomicSub(active, 1);
        if (before == 1 && use_cond) cudaGraphSetConditional(cond, 0);
      }
    }
  }
  if (threadIdx.x != 0 || !use_cond) return;
  if (refine) atomicOr(&flags[0], 1u);
  __threadfence();
  if (atomicAdd(&flags[1], 1u) == gridDim.x - 1) {  // last block of the class
    __threadfence();
    const unsigned any = atomicExch(&flags[0], 0u);
    flags[1] = 0;
    cudaGraphSetConditional(if_cond, any ? 1u : 0u);
  }
}

// FP64 refinement per slab (k_mx_outer with slab ends): mode 0 residual of
// Psi[cur] for every slab; mode 1 for slabs that asked for it: Psi[cur^1] =
// Psi[cur] + delta[dcur] and, unless the slab is done, its residual.
// hwcvt = 0: integer-pipe conversions and in-tile upstream neighbours read back
// from Psi[cur^1], as in k_mx_outer; hwcvt = 1: compiler conversions (same bits).
__global__ void __launch_bounds__(256) k_b_mx_outer(BatchClassDev c, const DevState *__restrict__ ds, int mode,
                                                    int hwcvt) {
  extern __shared__ double smd[];
  const int CB = blockDim.x, N = c.N, G = c.G, Jc = c.Jc;
  const int cl = threadIdx.x, g = threadIdx.y;
  const int N2 = N / 2;
  for (int s = 0; s < c.n_slabs; s++) {
    if (mode == 1 && !ds[s].refine) continue;  // uniform
    if (mode == 0 && ds[s].done) continue;
    const bool apply = mode != 0;
    const bool resid = mode == 0 || !ds[s].done;
    const bool reuse = apply && !hwcvt;
    const int cur = ds[s].cur;
    const double *__restrict__ Pin = cur ? c.Psi1 : c.Psi0;
    double *__restrict__ Pout = cur ? c.Psi0 : c.Psi1;
    const float *__restrict__ Dl = ds[s].dcur ? c.D1 : c.D0;
    const double *inc = c.inc + (size_t)s * 2 * G * N * 2;
    const int t0 = c.slab_tile0[s], t1 = c.slab_tile1[s];
    const int G_ = gridDim.x;
    const int first = t0 + (((int)blockIdx.x - t0 % G_) % G_ + G_) % G_;
    for (int tile = first; tile < t1; tile += G_) {
      const int j = c.tile_first_cell[tile] + cl;
      const int jl = j - c.slab_start[s];
      const int Js = c.slab_J[s];
      const bool active = jl < Js;
      const int tau = active ? c.type[j] : 0;
      double ph[4] = {0.0, 0.0, 0.0, 0.0};
      if (active) {
        for (int m = 0; m < N; m++) {
          const int gm = g * N + m;
          const size_t base = (size_t)gm * 4 * Jc + j;
          const double wm = c.w[m];
#pragma unroll
          for (int p = 0; p < 4; p++) {
            double v = Pin[base + (size_t)p * Jc];
            if (apply) {
              v += cvt_f2d(hwcvt, Dl[base + (size_t)p * Jc]);
              Pout[base + (size_t)p * Jc] = v;
            }
            ph[p] = fma(wm, v, ph[p]);
          }
        }
      }
      if (!resid) continue;  // uniform over the block
      double *ph_s = smd;
      __syncthreads();
#pragma unroll
      for (int p = 0; p < 4; p++) ph_s[(size_t)(g * 4 + p) * CB + cl] = ph[p];
      __syncthreads();
      if (!active) continue;
      double sv[4] = {0.0, 0.0, 0.0, 0.0};
      for (int gp = 0; gp < G; gp++) {
        const double k = c.Kap[((size_t)tau * G + gp) * G + g];
#pragma unroll
        for (int p = 0; p < 4; p++) sv[p] = fma(k, ph_s[(size_t)(gp * 4 + p) * CB + cl], sv[p]);
      }
      const double *P = apply ? Pout : Pin;  // Pout: written by this block before the barrier
      for (int m = 0; m < N; m++) {
        const int gm = g * N + m;
        const size_t base = (size_t)gm * 4 * Jc + j;
        const double v0 = P[base], v1 = P[base + (size_t)Jc], v2 = P[base + 2 * (size_t)Jc],
                     v3 = P[base + 3 * (size_t)Jc];
        const double *L = c.Lco + ((size_t)tau * G * N + gm) * 5;
        const double a = L[0], hm = L[1], ha = L[2], al = L[3], aa = L[4];
        double r0 = c.cvec[base] + sv[0];
        double r1 = c.cvec[base + (size_t)Jc] + sv[1];
        double r2 = c.cvec[base + 2 * (size_t)Jc] + sv[2];
        double r3 = c.cvec[base + 3 * (size_t)Jc] + sv[3];
        if (m >= N2) {
          double uk, uh;
          if (jl > 0) {
            const size_t nb = base - 1;
            if (reuse && cl > 0) {
              uk = Pout[nb + (size_t)Jc];
              uh = Pout[nb + 3 * (size_t)Jc];
            } else {
              uk = Pin[nb + (size_t)Jc];
              uh = Pin[nb + 3 * (size_t)Jc];
              if (apply) {
                uk += cvt_f2d(hwcvt, Dl[nb + (size_t)Jc]);
                uh += cvt_f2d(hwcvt, Dl[nb + 3 * (size_t)Jc]);
              }
            }
          } else {
            uk = inc[gm * 2 + 0];
            uh = inc[gm * 2 + 1];
          }
          r0 = fma(c.mu[m], uk, r0);
          r2 = fma(c.mu[m], uh, r2);
        } else {
          double uk, uh;
          if (jl < Js - 1) {
            const size_t nb = base + 1;
            if (reuse && cl < CB - 1) {
              uk = Pout[nb];
              uh = Pout[nb + 2 * (size_t)Jc];
            } else {
              uk = Pin[nb];
              uh = Pin[nb + 2 * (size_t)Jc];
              if (apply) {
                uk += cvt_f2d(hwcvt, Dl[nb]);
                uh += cvt_f2d(hwcvt, Dl[nb + 2 * (size_t)Jc]);
              }
            }
          } else {
            uk = inc[(G * N + gm) * 2 + 0];
            uh = inc[(G * N + gm) * 2 + 1];
          }
          r1 = fma(-c.mu[m], uk, r1);
          r3 = fma(-c.mu[m], uh, r3);
        }
        r0 = fma(-a, v0, fma(-hm, v1, fma(-ha, v2, r0)));
        r1 = fma(hm, v0, fma(-a, v1, fma(-ha, v3, r1)));
        r2 = fma(al, v0, fma(-aa, v2, fma(-hm, v3, r2)));
        r3 = fma(al, v1, fma(hm, v2, fma(-aa, v3, r3)));
        const float f0 = cvt_d2f(hwcvt, r0), f1 = cvt_d2f(hwcvt, r1), f2 = cvt_d2f(hwcvt, r2), f3 = cvt_d2f(hwcvt, r3);
        const float *Li = c.Linv32 + ((size_t)tau * G * N + gm) * 16;
#pragma unroll
        for (int p = 0; p < 4; p++)
          c.z32[base + (size_t)p * Jc] =
              fmaf(Li[p * 4 + 3], f3, fmaf(Li[p * 4 + 2], f2, fmaf(Li[p * 4 + 1], f1, Li[p * 4 + 0] * f0)));
      }
    }
  }
}

// After the loop: settle a refinement made by the last body (flip Psi, zero correction).
__global__ void k_b_mx_settle(int n_slabs, DevState *ds) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slabs) return;
  if (ds[s].refine) {
    ds[s].cur ^= 1;
    ds[s].refine = 0;
    ds[s].blk_i = 0;
  }
}

// ---------------------------------------------------------------- register form
// The same sweep with the angles of a cell split over P = N/NP threads, each
// keeping its NP angles' t = tc + Cin u in registers (no per-angle staging in
// shared memory, so large N*G no longer limits the block to a few cells).
// Block = CB cells x (G*P) threads; the angle sum y is reduced across the
// chunks in a fixed order, then the (4G x 4G) apply s = Mp y is split over the
// chunk threads of each group.  MX = false: the FP64 sweep (Psi ping-pong,
// incident flux at slab ends); MX = true: the FP32 correction sweep of the mixed
// form (delta ping-pong, zero inflow at slab ends, zero input on a new block).
template <typename T>
struct BRegIO;
template <>
struct BRegIO<double> {
  __device__ static const double *base(const BatchClassDev &c) { return c.tc; }
  __device__ static const double *cin(const BatchClassDev &c) { return c.Cin; }
  __device__ static const double *linv(const BatchClassDev &c) { return c.Linv; }
  __device__ static const double *mp(const BatchClassDev &c) { return c.Mp; }
  __device__ static const double *w(const BatchClassDev &c) { return c.w; }
  __device__ static double fm(double a, double b, double x) { return fma(a, b, x); }
};
template <>
struct BRegIO<float> {
  __device__ static const float *base(const BatchClassDev &c) { return c.z32; }
  __device__ static const float *cin(const BatchClassDev &c) { return c.Cin32; }
  __device__ static const float *linv(const BatchClassDev &c) { return c.Linv32; }
  __device__ static const float *mp(const BatchClassDev &c) { return c.Mp32; }
  __device__ static const float *w(const BatchClassDev &c) { return c.w32; }
  __device__ static float fm(float a, float b, float x) { return fmaf(a, b, x); }
};

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_b_sweep_reg(BatchClassDev c, const DevState *__restrict__ ds) {
  using IO = BRegIO<T>;
  constexpr bool MX = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[8];
  const int CB = blockDim.x, N = c.N, G = c.G, Jc = c.Jc;
  const int P = N / NP;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int G4 = 4 * G;
  T *y_s = (T *)smraw;                      // [G*P*4][CB] chunk partials of y
  T *yr_s = y_s + (size_t)G * P * 4 * CB;   // [4G][CB] y
  T *s_s = yr_s + (size_t)G4 * CB;          // [4G][CB] s = Mp y
  const int N2 = N / 2;
  const T *__restrict__ Bv = IO::base(c);
  const T *__restrict__ Cin = IO::cin(c);
  const T *__restrict__ Linv = IO::linv(c);
  const T *__restrict__ Mp = IO::mp(c);
  const T *__restrict__ w = IO::w(c);
  const int tid = threadIdx.y * CB + threadIdx.x;
  const int nthr = CB * G * P;
  for (int s = 0; s < c.n_slabs; s++) {
    if (ds[s].done) continue;  // uniform over the block
    bool zero = false;
    const T *In;
    T *Out;
    if (MX) {
      zero = ds[s].refine || ds[s].blk_i == 0;
      const int dc = ds[s].dcur;
      In = (const T *)(dc ? (const void *)c.D1 : (const void *)c.D0);
      Out = (T *)(dc ? (void *)c.D0 : (void *)c.D1);
    } else {
      const int cur = ds[s].cur;
      In = (const T *)(cur ? (const void *)c.Psi1 : (const void *)c.Psi0);
      Out = (T *)(cur ? (void *)c.Psi0 : (void *)c.Psi1);
    }
    const double *inc = c.inc + (size_t)s * 2 * G * N * 2;
    const int t0 = c.slab_tile0[s], t1 = c.slab_tile1[s];
    const int Gd = gridDim.x;
    const int first = t0 + (((int)blockIdx.x - t0 % Gd) % Gd + Gd) % Gd;
    const int s0c = c.slab_start[s], Js = c.slab_J[s];
    for (int tile = first; tile < t1; tile += Gd) {
      const int j = c.tile_first_cell[tile] + cl;
      const int jl = j - s0c;
      const bool active = jl < Js;
      const int tau = active ? c.type[j] : 0;
      const size_t tb = (size_t)tau * G * N;
      T t[NP][4];
      T y0 = T(0), y1 = T(0), y2 = T(0), y3 = T(0);
      if (active) {
#pragma unroll
        for (int i = 0; i < NP; i++) {
          const int m = m0 + i;
          const int gm = g * N + m;
          const size_t base = (size_t)gm * 4 * Jc + j;
          T uk = T(0), uh = T(0);
          if (m >= N2) {
            if (jl > 0) {
              if (!zero) {
                uk = In[base + (size_t)Jc - 1];
                uh = In[base + 3 * (size_t)Jc - 1];
              }
            } else if (!MX) {
              uk = (T)inc[gm * 2 + 0];
              uh = (T)inc[gm * 2 + 1];
            }
          } else {
            if (jl < Js - 1) {
              if (!zero) {
                uk = In[base + 1];
                uh = In[base + 2 * (size_t)Jc + 1];
              }
            } else if (!MX) {
              uk = (T)inc[(G * N + gm) * 2 + 0];
              uh = (T)inc[(G * N + gm) * 2 + 1];
            }
          }
          const T *C = Cin + (tb + gm) * 8;
          t[i][0] = IO::fm(C[1], uh, IO::fm(C[0], uk, Bv[base]));
          t[i][1] = IO::fm(C[3], uh, IO::fm(C[2], uk, Bv[base + (size_t)Jc]));
          t[i][2] = IO::fm(C[5], uh, IO::fm(C[4], uk, Bv[base + 2 * (size_t)Jc]));
          t[i][3] = IO::fm(C[7], uh, IO::fm(C[6], uk, Bv[base + 3 * (size_t)Jc]));
          const T wm = w[m];
          y0 = IO::fm(wm, t[i][0], y0);
          y1 = IO::fm(wm, t[i][1], y1);
          y2 = IO::fm(wm, t[i][2], y2);
          y3 = IO::fm(wm, t[i][3], y3);
        }
      }
      {
        T *ys = y_s + (size_t)(gy * 4) * CB + cl;
        ys[0] = y0;
        ys[CB] = y1;
        ys[2 * CB] = y2;
        ys[3 * CB] = y3;
      }
      __syncthreads();
      // y_{g,q} = sum over the group's chunks (fixed order)
      for (int q = ch; q < 4; q += P) {
        T v = y_s[(size_t)((g * P) * 4 + q) * CB + cl];
        for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * CB + cl];
        yr_s[(size_t)(g * 4 + q) * CB + cl] = v;
      }
      __syncthreads();
      // s_{g,q} = sum_k Mp[g*4+q][k] y_k
      if (active) {
        for (int q = ch; q < 4; q += P) {
          const T *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
          T v = T(0);
          for (int k = 0; k < G4; k++) v = IO::fm(M[k], yr_s[(size_t)k * CB + cl], v);
          s_s[(size_t)(g * 4 + q) * CB + cl] = v;
        }
      }
      __syncthreads();
      T e2 = T(0);
      if (active) {
        const T sv0 = s_s[(size_t)(g * 4 + 0) * CB + cl], sv1 = s_s[(size_t)(g * 4 + 1) * CB + cl];
        const T sv2 = s_s[(size_t)(g * 4 + 2) * CB + cl], sv3 = s_s[(size_t)(g * 4 + 3) * CB + cl];
#pragma unroll
        for (int i = 0; i < NP; i++) {
          const int gm = g * N + m0 + i;
          const size_t base = (size_t)gm * 4 * Jc + j;
          const T *L = Linv + (tb + gm) * 16;
#pragma unroll
          for (int p = 0; p < 4; p++) {
            const T o = IO::fm(L[p * 4 + 3], sv3,
                               IO::fm(L[p * 4 + 2], sv2, IO::fm(L[p * 4 + 1], sv1, IO::fm(L[p * 4 + 0], sv0, t[i][p]))));
            const T d = zero ? o : o - In[base + (size_t)p * Jc];
            e2 = IO::fm(d, d, e2);
            Out[base + (size_t)p * Jc] = o;
          }
        }
      }
      double v = (double)e2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double acc = 0.0;
        for (int i = 0; i < (nthr + 31) / 32; i++) acc += red[i];
        c.partials[tile] = acc;
      }
      // the next tile's first shared-memory writes come after the y_s barrier;
      // red is rewritten only after two more barriers
    }
  }
}

// ---------------------------------------------------------------- launches
size_t b_sweep_smem(int N, int G, int cb) {
  return (size_t)cb * ((size_t)G * N * 4 * 8 + (size_t)G * 4 * 8);
}

void launch_b_step_const(BatchClass &c, cudaStream_t st) {
  dim3 grid((c.d.Jc + 255) / 256, c.d.G * c.d.N);
  k_b_step_const<<<grid, 256, 0, st>>>(c.d.Jc, c.d.N, c.d.G, c.d.type, c.d.seg, c.d.tdx, c.d.tah, c.d.Q,
                                       c.d.psi_prev, c.d.Linv, c.d.tc);
}

size_t b_reg_smem(int N, int G, int cb, int np, int es) {
  const int P = N / np;
  return (size_t)cb * ((size_t)G * P * 4 + 8 * (size_t)G) * es;
}

template <typename T>
static const void *reg_kernel(int np) {
  switch (np) {
    case 2: return (const void *)k_b_sweep_reg<T, 2>;
    case 4: return (const void *)k_b_sweep_reg<T, 4>;
    case 8: return (const void *)k_b_sweep_reg<T, 8>;
    default: return nullptr;
  }
}
const void *k_b_reg_ptr(int np, bool mixed) { return mixed ? reg_kernel<float>(np) : reg_kernel<double>(np); }

template <typename T>
static void launch_reg(BatchClass &c, const DevState *ds, cudaStream_t st) {
  const int P = c.d.N / c.np;
  dim3 block(c.cb, c.d.G * P);
  const size_t smem = b_reg_smem(c.d.N, c.d.G, c.cb, c.np, (int)sizeof(T));
  switch (c.np) {
    case 2: k_b_sweep_reg<T, 2><<<c.grid, block, smem, st>>>(c.d, ds); break;
    case 4: k_b_sweep_reg<T, 4><<<c.grid, block, smem, st>>>(c.d, ds); break;
    case 8: k_b_sweep_reg<T, 8><<<c.grid, block, smem, st>>>(c.d, ds); break;
    default: break;
  }
}

void launch_b_sweep(BatchClass &c, DevState *ds, cudaStream_t st) {
  if (c.np) {
    launch_reg<double>(c, ds, st);
    return;
  }
  dim3 block(c.cb, c.d.G);
  k_b_sweep<<<c.grid, block, b_sweep_smem(c.d.N, c.d.G, c.cb), st>>>(c.d, ds);
}

void launch_b_finalize(BatchClass &c, DevState *ds, int *active, int use_cond, cudaGraphConditionalHandle cond,
                       cudaStream_t st) {
  k_b_finalize<<<c.d.n_slabs, kBFinThreads, 0, st>>>(c.d, ds, active, use_cond, cond);
}

void launch_b_carry(BatchClass &c, DevState *ds, cudaStream_t st) {
  k_b_carry<<<c.d.Jc / 32, dim3(32, c.d.G), 0, st>>>(c.d, ds);
  k_b_balance_final<<<dim3(c.d.n_slabs, c.d.G), 32, 0, st>>>(c.d, ds);
}

const void *k_b_sweep_ptr() { return (const void *)k_b_sweep; }
const void *k_b_mx_inner_ptr() { return (const void *)k_b_mx_inner; }

size_t b_mx_smem(int N, int G, int cb) { return (size_t)cb * ((size_t)G * N * 4 + (size_t)G * 4) * 4; }

void launch_b_mx_step_const(BatchClass &c, cudaStream_t st) {
  dim3 grid((c.d.Jc + 255) / 256, c.d.G * c.d.N);
  k_b_mx_step_const<<<grid, 256, 0, st>>>(c.d);
}

void launch_b_mx_inner(BatchClass &c, DevState *ds, cudaStream_t st) {
  if (c.np) {
    launch_reg<float>(c, ds, st);
    return;
  }
  k_b_mx_inner<<<c.grid, dim3(c.cb, c.d.G), b_mx_smem(c.d.N, c.d.G, c.cb), st>>>(c.d, ds);
}

void launch_b_mx_finalize(BatchClass &c, DevState *ds, int *active, int use_cond, cudaGraphConditionalHandle cond,
                          cudaStream_t st) {
  k_b_mx_finalize<<<c.d.n_slabs, kBFinThreads, 0, st>>>(c.d, ds, active, use_cond, cond, c.if_flags,
                                                         (cudaGraphConditionalHandle)c.if_handle);
}

void launch_b_mx_outer(BatchClass &c, DevState *ds, int mode, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(c.d.n_tiles, 4 * sms);
  const char *cv = hook_env("OCI_MX_OUTER_CVT");  // "hw": compiler conversions
  const int hwcvt = (cv && cv[0] == 'h') ? 1 : 0;
  k_b_mx_outer<<<grid > 0 ? grid : 1, dim3(c.cb, c.d.G), (size_t)c.cb * c.d.G * 4 * sizeof(double), st>>>(c.d, ds,
                                                                                                         mode, hwcvt);
}

void launch_b_mx_settle(BatchClass &c, DevState *ds, cudaStream_t st) {
  k_b_mx_settle<<<(c.d.n_slabs + 127) / 128, 128, 0, st>>>(c.d.n_slabs, ds);
}

int b_max_grid(int N, int G, int cb) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_b_sweep, cb * G, b_sweep_smem(N, G, cb));
  return sms * (per > 0 ? per : 1);
}

int b_reg_max_grid(int N, int G, int cb, int np, bool mixed) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_b_reg_ptr(np, mixed), cb * G * (N / np),
                                                b_reg_smem(N, G, cb, np, mixed ? 4 : 8));
  return sms * (per > 0 ? per : 1);
}

int b_mx_max_grid(int N, int G, int cb) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_b_mx_inner, cb * G, b_mx_smem(N, G, cb));
  return sms * (per > 0 ? per : 1);
}

}  // namespace oci
