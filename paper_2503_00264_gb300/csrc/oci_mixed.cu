// oci_mixed.cu -- mixed-precision form of the OCI step: inner sweeps on an FP32
// correction, FP64 refinement.
//
// With A = L_c - S block diagonal and B the lagged-inflow coupling (Eq. oci),
// plain OCI is Psi^{l+1} = A^{-1}(c + B Psi^l).  From an outer iterate Psi with
// FP64 residual r = c + B Psi - A Psi, the iterates of plain OCI are
// Psi^{l+i} = Psi + delta^i with
//     delta^0 = 0,   delta^{i+1} = A^{-1}(r + B delta^i),
// and the per-sweep change e_i = ||delta^{i+1} - delta^i||_2 equals plain OCI's
// ||Psi^{l+i+1} - Psi^{l+i}||_2.  The inner recursion runs in FP32 (structured
// cell solve with FP32 tables); every few sweeps the correction is folded into
// the FP64 iterate and the residual is recomputed in FP64, which removes the
// FP32 error accumulated so far (defect correction).  The stop rule of Sec. 2.1
// is applied to every inner sweep, so sweep counts track the FP64 form.
//
// A refinement happens after k_max inner sweeps, or once e < theta * (first e
// of the block) -- by then the FP32 correction has gained about -log10(theta)
// digits and more inner sweeps would only resolve FP32 rounding -- and at
// convergence.  The stop rule is accepted only on a sweep whose correction is
// small (first sweep after a refinement, or a block that began below tol), so
// the committed iterate carries no more than low-precision rounding of a tiny
// correction; this costs at most one extra sweep per step.  FP64 is kept for Psi,
// the residual, the norm accumulation, the balance tallies and the carry.
#include <cuda.h>
#include <math.h>

#include "oci_cvt.cuh"
#include "oci_device.cuh"
#include "oci_mixed_dev.cuh"

namespace oci {

// Index of row r, cell j of an FP32 correction array: [R][Jp] (tsh = 0) or
// tile-major [J/T][R][T] with T = 2^(tsh & 0xff); with bit 0x100 the columns of
// a tile are ordered by colour (even cells, then odd cells: red-black form).
__device__ __forceinline__ size_t fidx(int tsh, int R, size_t Jp, int r, int j) {
  if (!tsh) return (size_t)r * Jp + j;
  const int sh = tsh & 0xff;
  int c = j & ((1 << sh) - 1);
  if (tsh & 0x100) c = (c & 1) * (1 << (sh - 1)) + (c >> 1);
  return ((((size_t)(j >> sh)) * R + r) << sh) + (size_t)c;
}


int mx_tile_shift(const Handle &h) {
  const int sh = h.mx_cb == 16 ? 4 : h.mx_cb == 32 ? 5 : h.mx_cb == 64 ? 6 : 7;
  if (h.mx_kind == kMxTiled || h.mx_kind == kMxTiledP || h.mx_kind == kMxTiledB || h.mx_kind == kMxTiled2 ||
      h.mx_kind == kMxTiled2Occ || h.mx_kind == kMxWarp2)
    return sh;
  if (h.mx_kind == kMxRB || h.mx_kind == kMxRB2) return sh | 0x100;
  return 0;
}

// ---------------------------------------------------------------- inner sweep
// delta_out = A~^{-1}(r + B delta_in) through the structured solve in FP32:
// t = z + Cin u, y = sum_m w t, s = Mp y, delta = t + Linv s, where z = A~-block
// solve of r precomputed by the outer kernel (z = Linv r).  The correction has
// zero incident flux at the slab ends (the boundary values live in r).
__global__ void __launch_bounds__(256) k_mx_inner(int J, int Jp, int N, int G, int P,
                                                  const int32_t *__restrict__ type, const float *__restrict__ Linv,
                                                  const float *__restrict__ Cin, const float *__restrict__ Mp,
                                                  const float *__restrict__ w, const float *__restrict__ z, float *D0,
                                                  float *D1, DevState *ds, double *__restrict__ partials,
                                                  unsigned *counter, double *e_hist,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ float smf[];
  __shared__ double red[32];
  __shared__ bool s_last;
  const int CB = blockDim.x;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P;
  const int NP = N / P, m0 = ch * NP;
  const int j = blockIdx.x * CB + cl;
  if (ds->done) return;
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  float *t_s = smf;
  float *y_s = smf + (size_t)G * N * 4 * CB;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const int N2 = N / 2;
  const size_t tb = (size_t)tau * G * N;
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (active) {
#pragma unroll 4
    for (int m = m0; m < m0 + NP; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      float uk = 0.f, uh = 0.f;
      if (!zero) {
        if (m >= N2) {
          if (j > 0) {
            uk = Din[base + (size_t)Jp - 1];
            uh = Din[base + 3 * (size_t)Jp - 1];
          }
        } else if (j < J - 1) {
          uk = Din[base + 1];
          uh = Din[base + 2 * (size_t)Jp + 1];
        }
      }
      const float *C = Cin + (tb + gm) * 8;
      const float t0 = fmaf(C[1], uh, fmaf(C[0], uk, z[base]));
      const float t1 = fmaf(C[3], uh, fmaf(C[2], uk, z[base + (size_t)Jp]));
      const float t2 = fmaf(C[5], uh, fmaf(C[4], uk, z[base + 2 * (size_t)Jp]));
      const float t3 = fmaf(C[7], uh, fmaf(C[6], uk, z[base + 3 * (size_t)Jp]));
      float *ts = t_s + (size_t)(gm * 4) * CB + cl;
      ts[0] = t0;
      ts[CB] = t1;
      ts[2 * CB] = t2;
      ts[3 * CB] = t3;
      const float wm = w[m];
      y0 = fmaf(wm, t0, y0);
      y1 = fmaf(wm, t1, y1);
      y2 = fmaf(wm, t2, y2);
      y3 = fmaf(wm, t3, y3);
    }
    float *ys = y_s + (size_t)(gy * 4) * CB + cl;
    ys[0] = y0;
    ys[CB] = y1;
    ys[2 * CB] = y2;
    ys[3 * CB] = y3;
  }
  __syncthreads();
  float e2 = 0.f;
  if (active) {
    const int G4 = 4 * G;
    const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int k = 0; k < G4; k++) {
      const int gp = k >> 2, q = k & 3;
      float yk = y_s[(size_t)((gp * P) * 4 + q) * CB + cl];
      for (int c = 1; c < P; c++) yk += y_s[(size_t)((gp * P + c) * 4 + q) * CB + cl];
      s0 = fmaf(M[k], yk, s0);
      s1 = fmaf(M[G4 + k], yk, s1);
      s2 = fmaf(M[2 * G4 + k], yk, s2);
      s3 = fmaf(M[3 * G4 + k], yk, s3);
    }
#pragma unroll 4
    for (int m = m0; m < m0 + NP; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const float *L = Linv + (tb + gm) * 16;
      const float *ts = t_s + (size_t)(gm * 4) * CB + cl;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float o = fmaf(L[p * 4 + 3], s3, fmaf(L[p * 4 + 2], s2, fmaf(L[p * 4 + 1], s1, fmaf(L[p * 4 + 0], s0, ts[p * CB]))));
        const float d = zero ? o : o - Din[base + (size_t)p * Jp];
        e2 = fmaf(d, d, e2);
        Dout[base + (size_t)p * Jp] = o;
      }
    }
  }
  // FP64 accumulation of the per-thread FP32 partial sums
  double v = (double)e2;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  // the block that finishes last reduces all partials and applies the stop rule
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

// ---------------------------------------------------------------- inner sweep, register form
// The same FP32 inner sweep with the N angles of a cell split over P = N/NP
// threads, each keeping its NP angles' t and delta_in in registers: all of a
// thread's loads (z, the upstream edges, its own delta_in for the norm) are
// issued before any arithmetic, so more bytes are in flight per SM than in the
// staged form.  The angle sum y is reduced over the chunks in a fixed order and
// s = Mp y is split over the chunk threads of each group.
size_t mx_reg_smem(int G, int cb, int P) { return (size_t)cb * ((size_t)G * P * 4 + 8 * (size_t)G) * 4; }

template <int NP>
__global__ void __launch_bounds__(256) k_mx_inner_reg(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                                      const float *__restrict__ Linv, const float *__restrict__ Cin,
                                                      const float *__restrict__ Mp, const float *__restrict__ w,
                                                      const float *__restrict__ z, float *D0, float *D1,
                                                      DevState *ds, double *__restrict__ partials,
                                                      unsigned *counter, double *e_hist,
                                                      cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ float smr[];
  __shared__ double red[8];
  __shared__ bool s_last;
  const int CB = blockDim.x, P = N / NP, G4 = 4 * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int j = blockIdx.x * CB + cl;
  if (ds->done) return;  // uniform across the grid
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  float *y_s = smr;                          // [G*P*4][CB] chunk partials of y
  float *yr_s = y_s + (size_t)G * P * 4 * CB;  // [4G][CB] y
  float *s_s = yr_s + (size_t)G4 * CB;        // [4G][CB] s
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const int N2 = N / 2;
  const size_t tb = (size_t)tau * G * N;
  float t[NP][4], old[NP][4];
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (active) {
    float uk[NP], uh[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const size_t base = (size_t)(g * N + m) * 4 * Jp + j;
      uk[i] = 0.f;
      uh[i] = 0.f;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        t[i][p] = z[base + (size_t)p * Jp];
        old[i][p] = 0.f;
      }
      if (!zero) {
#pragma unroll
        for (int p = 0; p < 4; p++) old[i][p] = Din[base + (size_t)p * Jp];
        if (m >= N2) {
          if (j > 0) {
            uk[i] = Din[base + (size_t)Jp - 1];
            uh[i] = Din[base + 3 * (size_t)Jp - 1];
          }
        } else if (j < J - 1) {
          uk[i] = Din[base + 1];
          uh[i] = Din[base + 2 * (size_t)Jp + 1];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const float *C = Cin + (tb + g * N + m) * 8;
#pragma unroll
      for (int p = 0; p < 4; p++) t[i][p] = fmaf(C[2 * p + 1], uh[i], fmaf(C[2 * p], uk[i], t[i][p]));
      const float wm = w[m];
      y0 = fmaf(wm, t[i][0], y0);
      y1 = fmaf(wm, t[i][1], y1);
      y2 = fmaf(wm, t[i][2], y2);
      y3 = fmaf(wm, t[i][3], y3);
    }
  }
  {
    float *ys = y_s + (size_t)(gy * 4) * CB + cl;
    ys[0] = y0;
    ys[CB] = y1;
    ys[2 * CB] = y2;
    ys[3 * CB] = y3;
  }
  __syncthreads();
  for (int q = ch; q < 4; q += P) {  // y_{g,q}: fixed-order sum over the group's chunks
    float v = y_s[(size_t)((g * P) * 4 + q) * CB + cl];
    for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * CB + cl];
    yr_s[(size_t)(g * 4 + q) * CB + cl] = v;
  }
  __syncthreads();
  if (active)
    for (int q = ch; q < 4; q += P) {  // s_{g,q} = sum_k Mp[g*4+q][k] y_k
      const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
      float v = 0.f;
      for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[(size_t)k * CB + cl], v);
      s_s[(size_t)(g * 4 + q) * CB + cl] = v;
    }
  __syncthreads();
  float e2 = 0.f;
  if (active) {
    const float s0 = s_s[(size_t)(g * 4 + 0) * CB + cl], s1 = s_s[(size_t)(g * 4 + 1) * CB + cl];
    const float s2 = s_s[(size_t)(g * 4 + 2) * CB + cl], s3 = s_s[(size_t)(g * 4 + 3) * CB + cl];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int gm = g * N + m0 + i;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const float *L = Linv + (tb + gm) * 16;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float o = fmaf(L[p * 4 + 3], s3, fmaf(L[p * 4 + 2], s2, fmaf(L[p * 4 + 1], s1, fmaf(L[p * 4 + 0], s0, t[i][p]))));
        const float d = o - old[i][p];
        e2 = fmaf(d, d, e2);
        Dout[base + (size_t)p * Jp] = o;
      }
    }
  }
  // FP64 accumulation of the per-thread FP32 partial sums
  double v = (double)e2;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

// ---------------------------------------------------------------- inner sweep, tiled layout
// The register form on the tile-major FP32 layout [J/T][4NG][T] (T cells per
// tile, one tile per block): all rows of a thread's angles are at fixed
// offsets (i*4 + p)*T from one base pointer, so the loads and stores need no
// per-element address arithmetic, and a tile's operands are contiguous in HBM.
// The per-type tables are fetched as float4.  Neighbour edges across a tile
// boundary come from the adjacent tile's first / last column.
size_t mx_tiled_smem(int G, int T, int P) { return mx_reg_smem(G, T, P); }

template <int T, int NP>
__global__ void __launch_bounds__(256) k_mx_inner_tiled(int J, int N, int G, const int32_t *__restrict__ type,
                                                        const float *__restrict__ Linv,
                                                        const float *__restrict__ Cin, const float *__restrict__ Mp,
                                                        const float *__restrict__ w, const float *__restrict__ z,
                                                        float *D0, float *D1, DevState *ds,
                                                        double *__restrict__ partials, unsigned *counter,
                                                        double *e_hist, cudaGraphConditionalHandle cond,
                                                        int use_cond) {
  extern __shared__ float smr[];
  __shared__ double red[8];
  __shared__ bool s_last;
  const int P = N / NP, G4 = 4 * G, R = 4 * N * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int j = blockIdx.x * T + cl;
  if (ds->done) return;  // uniform across the grid
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  float *y_s = smr;
  float *yr_s = y_s + (size_t)G * P * 4 * T;
  float *s_s = yr_s + (size_t)G4 * T;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const int N2 = N / 2;
  const size_t tb = (size_t)tau * G * N;
  const size_t off = ((size_t)blockIdx.x * R + (size_t)(g * N + m0) * 4) * T + cl;
  const float *__restrict__ zb = z + off;
  const float *__restrict__ db = Din + off;
  float *__restrict__ ob = Dout + off;
  float t[NP][4], old[NP][4];
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (active) {
    float uk[NP], uh[NP];
    // upstream cell j-1 / j+1: same tile, or the last / first column of the adjacent tile
    const long long offL = cl > 0 ? -1 : (T - 1) - (long long)R * T;
    const long long offR = cl < T - 1 ? 1 : (long long)R * T - (T - 1);
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        t[i][p] = zb[(i * 4 + p) * T];
        old[i][p] = zero ? 0.f : db[(i * 4 + p) * T];
      }
      uk[i] = 0.f;
      uh[i] = 0.f;
      if (!zero) {
        if (m >= N2) {
          if (j > 0) {
            uk[i] = db[offL + (i * 4 + 1) * T];
            uh[i] = db[offL + (i * 4 + 3) * T];
          }
        } else if (j < J - 1) {
          uk[i] = db[offR + (i * 4 + 0) * T];
          uh[i] = db[offR + (i * 4 + 2) * T];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const float4 *C4 = reinterpret_cast<const float4 *>(Cin + (tb + g * N + m) * 8);
      const float4 ca = C4[0], cb = C4[1];
      t[i][0] = fmaf(ca.y, uh[i], fmaf(ca.x, uk[i], t[i][0]));
      t[i][1] = fmaf(ca.w, uh[i], fmaf(ca.z, uk[i], t[i][1]));
      t[i][2] = fmaf(cb.y, uh[i], fmaf(cb.x, uk[i], t[i][2]));
      t[i][3] = fmaf(cb.w, uh[i], fmaf(cb.z, uk[i], t[i][3]));
      const float wm = w[m];
      y0 = fmaf(wm, t[i][0], y0);
      y1 = fmaf(wm, t[i][1], y1);
      y2 = fmaf(wm, t[i][2], y2);
      y3 = fmaf(wm, t[i][3], y3);
    }
  }
  {
    float *ys = y_s + (size_t)(gy * 4) * T + cl;
    ys[0] = y0;
    ys[T] = y1;
    ys[2 * T] = y2;
    ys[3 * T] = y3;
  }
  __syncthreads();
  for (int q = ch; q < 4; q += P) {
    float v = y_s[(size_t)((g * P) * 4 + q) * T + cl];
    for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * T + cl];
    yr_s[(size_t)(g * 4 + q) * T + cl] = v;
  }
  __syncthreads();
  if (active)
    for (int q = ch; q < 4; q += P) {
      const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
      float v = 0.f;
      for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[(size_t)k * T + cl], v);
      s_s[(size_t)(g * 4 + q) * T + cl] = v;
    }
  __syncthreads();
  float e2 = 0.f;
  if (active) {
    const float s0 = s_s[(size_t)(g * 4 + 0) * T + cl], s1 = s_s[(size_t)(g * 4 + 1) * T + cl];
    const float s2 = s_s[(size_t)(g * 4 + 2) * T + cl], s3 = s_s[(size_t)(g * 4 + 3) * T + cl];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const float4 *L4 = reinterpret_cast<const float4 *>(Linv + (tb + g * N + m0 + i) * 16);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float4 L = L4[p];
        const float o = fmaf(L.w, s3, fmaf(L.z, s2, fmaf(L.y, s1, fmaf(L.x, s0, t[i][p]))));
        const float d = o - old[i][p];
        e2 = fmaf(d, d, e2);
        ob[(i * 4 + p) * T] = o;
      }
    }
  }
  double v = (double)e2;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

// ---------------------------------------------------------------- inner sweep, tiled + persistent
// The tiled register sweep as a persistent kernel: each block reads the device
// state once, stages the per-type tables (Linv, Cin, w, Mp) in shared memory
// when they fit (else reads them from global memory through the same generic
// pointers), walks the tiles tile = blockIdx.x, blockIdx.x + gridDim.x, ...
// and publishes one partial of the norm (its tiles summed in a fixed order).
// This removes the per-tile state read, table latency and end-of-block fence
// and atomic of the one-tile-per-block form.
size_t mx_tables_floats(const Handle &h) {
  const size_t T = h.tt.n_types, G = h.G, N = h.N;
  return T * G * N * 24 + N + T * 16 * G * G;
}
size_t mx_tp_smem(const Handle &h, int T, int P, bool stage) {
  return mx_reg_smem(h.G, T, P) + (stage ? mx_tables_floats(h) * 4 + 16 : 0);
}


// One tile of the tiled register sweep by the whole block; returns this
// thread's sum of squared changes.  Contains three block barriers; shared
// memory y_s / yr_s / s_s may be reused by the next call.
template <int T, int NP>
__device__ __forceinline__ float tiled_tile(int tile, int J, int N, int G, int cl, int gy, bool zero,
                                            const int32_t *__restrict__ type, const float *Linv, const float *Cin,
                                            const float *Mp, const float *w, const float *__restrict__ z,
                                            const float *__restrict__ Din, float *__restrict__ Dout, float *y_s,
                                            float *yr_s, float *s_s) {
  const int P = N / NP, G4 = 4 * G, R = 4 * N * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int N2 = N / 2;
  const long long offL = cl > 0 ? -1 : (T - 1) - (long long)R * T;
  const long long offR = cl < T - 1 ? 1 : (long long)R * T - (T - 1);
  const int j = tile * T + cl;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const size_t tb = (size_t)tau * G * N;
  const size_t off = ((size_t)tile * R + (size_t)(g * N + m0) * 4) * T + cl;
  const float *__restrict__ zb = z + off;
  const float *__restrict__ db = Din + off;
  float *__restrict__ ob = Dout + off;
  float t[NP][4], old[NP][4];
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (active) {
    float uk[NP], uh[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        t[i][p] = zb[(i * 4 + p) * T];
        old[i][p] = zero ? 0.f : db[(i * 4 + p) * T];
      }
      uk[i] = 0.f;
      uh[i] = 0.f;
      if (!zero) {
        if (m >= N2) {
          if (j > 0) {
            uk[i] = db[offL + (i * 4 + 1) * T];
            uh[i] = db[offL + (i * 4 + 3) * T];
          }
        } else if (j < J - 1) {
          uk[i] = db[offR + (i * 4 + 0) * T];
          uh[i] = db[offR + (i * 4 + 2) * T];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const float4 *C4 = reinterpret_cast<const float4 *>(Cin + (tb + g * N + m) * 8);
      const float4 ca = C4[0], cb = C4[1];
      t[i][0] = fmaf(ca.y, uh[i], fmaf(ca.x, uk[i], t[i][0]));
      t[i][1] = fmaf(ca.w, uh[i], fmaf(ca.z, uk[i], t[i][1]));
      t[i][2] = fmaf(cb.y, uh[i], fmaf(cb.x, uk[i], t[i][2]));
      t[i][3] = fmaf(cb.w, uh[i], fmaf(cb.z, uk[i], t[i][3]));
      const float wm = w[m];
      y0 = fmaf(wm, t[i][0], y0);
      y1 = fmaf(wm, t[i][1], y1);
      y2 = fmaf(wm, t[i][2], y2);
      y3 = fmaf(wm, t[i][3], y3);
    }
  }
  {
    float *ys = y_s + (size_t)(gy * 4) * T + cl;
    ys[0] = y0;
    ys[T] = y1;
    ys[2 * T] = y2;
    ys[3 * T] = y3;
  }
  __syncthreads();
  for (int q = ch; q < 4; q += P) {
    float v = y_s[(size_t)((g * P) * 4 + q) * T + cl];
    for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * T + cl];
    yr_s[(size_t)(g * 4 + q) * T + cl] = v;
  }
  __syncthreads();
  if (active)
    for (int q = ch; q < 4; q += P) {
      const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
      float v = 0.f;
      for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[(size_t)k * T + cl], v);
      s_s[(size_t)(g * 4 + q) * T + cl] = v;
    }
  __syncthreads();
  float e2 = 0.f;
  if (active) {
    const float s0 = s_s[(size_t)(g * 4 + 0) * T + cl], s1 = s_s[(size_t)(g * 4 + 1) * T + cl];
    const float s2 = s_s[(size_t)(g * 4 + 2) * T + cl], s3 = s_s[(size_t)(g * 4 + 3) * T + cl];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const float4 *L4 = reinterpret_cast<const float4 *>(Linv + (tb + g * N + m0 + i) * 16);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float4 L = L4[p];
        const float o = fmaf(L.w, s3, fmaf(L.z, s2, fmaf(L.y, s1, fmaf(L.x, s0, t[i][p]))));
        const float d = o - old[i][p];
        e2 = fmaf(d, d, e2);
        ob[(i * 4 + p) * T] = o;
      }
    }
  }
  // y_s of the next call is written only after the s_s barrier of this one;
  // s_s is rewritten two barriers later
  return e2;
}

// The tiled tile split in two for software pipelining across a block's tiles:
// tiled_load issues every global load of a tile into registers, tiled_compute
// does the rest (three block barriers, stores, the thread's squared change).
template <int NP>
struct TileRegs {
  float t[NP][4], old[NP][4], uk[NP], uh[NP];
  int tau;
  bool active;
};

template <int T, int NP>
__device__ __forceinline__ void tiled_load(TileRegs<NP> &r, int tile, int J, int N, int G, int cl, int gy, bool zero,
                                           const int32_t *__restrict__ type, const float *__restrict__ z,
                                           const float *__restrict__ Din) {
  const int P = N / NP, R = 4 * N * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int N2 = N / 2;
  const long long offL = cl > 0 ? -1 : (T - 1) - (long long)R * T;
  const long long offR = cl < T - 1 ? 1 : (long long)R * T - (T - 1);
  const int j = tile * T + cl;
  r.active = j < J;
  r.tau = r.active ? type[j] : 0;
  const size_t off = ((size_t)tile * R + (size_t)(g * N + m0) * 4) * T + cl;
  const float *__restrict__ zb = z + off;
  const float *__restrict__ db = Din + off;
#pragma unroll
  for (int i = 0; i < NP; i++) {
    const int m = m0 + i;
#pragma unroll
    for (int p = 0; p < 4; p++) {
      r.t[i][p] = r.active ? zb[(i * 4 + p) * T] : 0.f;
      r.old[i][p] = (r.active && !zero) ? db[(i * 4 + p) * T] : 0.f;
    }
    r.uk[i] = 0.f;
    r.uh[i] = 0.f;
    if (r.active && !zero) {
      if (m >= N2) {
        if (j > 0) {
          r.uk[i] = db[offL + (i * 4 + 1) * T];
          r.uh[i] = db[offL + (i * 4 + 3) * T];
        }
      } else if (j < J - 1) {
        r.uk[i] = db[offR + (i * 4 + 0) * T];
        r.uh[i] = db[offR + (i * 4 + 2) * T];
      }
    }
  }
}

template <int T, int NP>
__device__ __forceinline__ float tiled_compute(TileRegs<NP> &r, int tile, int N, int G, int cl, int gy,
                                               const float *Linv, const float *Cin, const float *Mp, const float *w,
                                               float *__restrict__ Dout, float *y_s, float *yr_s, float *s_s) {
  const int P = N / NP, G4 = 4 * G, R = 4 * N * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const size_t tb = (size_t)r.tau * G * N;
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (r.active) {
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const float4 *C4 = reinterpret_cast<const float4 *>(Cin + (tb + g * N + m) * 8);
      const float4 ca = C4[0], cb = C4[1];
      r.t[i][0] = fmaf(ca.y, r.uh[i], fmaf(ca.x, r.uk[i], r.t[i][0]));
      r.t[i][1] = fmaf(ca.w, r.uh[i], fmaf(ca.z, r.uk[i], r.t[i][1]));
      r.t[i][2] = fmaf(cb.y, r.uh[i], fmaf(cb.x, r.uk[i], r.t[i][2]));
      r.t[i][3] = fmaf(cb.w, r.uh[i], fmaf(cb.z, r.uk[i], r.t[i][3]));
      const float wm = w[m];
      y0 = fmaf(wm, r.t[i][0], y0);
      y1 = fmaf(wm, r.t[i][1], y1);
      y2 = fmaf(wm, r.t[i][2], y2);
      y3 = fmaf(wm, r.t[i][3], y3);
    }
  }
  {
    float *ys = y_s + (size_t)(gy * 4) * T + cl;
    ys[0] = y0;
    ys[T] = y1;
    ys[2 * T] = y2;
    ys[3 * T] = y3;
  }
  __syncthreads();
  for (int q = ch; q < 4; q += P) {
    float v = y_s[(size_t)((g * P) * 4 + q) * T + cl];
    for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * T + cl];
    yr_s[(size_t)(g * 4 + q) * T + cl] = v;
  }
  __syncthreads();
  if (r.active)
    for (int q = ch; q < 4; q += P) {
      const float *M = Mp + (size_t)r.tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
      float v = 0.f;
      for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[(size_t)k * T + cl], v);
      s_s[(size_t)(g * 4 + q) * T + cl] = v;
    }
  __syncthreads();
  float e2 = 0.f;
  if (r.active) {
    const float s0 = s_s[(size_t)(g * 4 + 0) * T + cl], s1 = s_s[(size_t)(g * 4 + 1) * T + cl];
    const float s2 = s_s[(size_t)(g * 4 + 2) * T + cl], s3 = s_s[(size_t)(g * 4 + 3) * T + cl];
    float *ob = Dout + ((size_t)tile * R + (size_t)(g * N + m0) * 4) * T + cl;
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const float4 *L4 = reinterpret_cast<const float4 *>(Linv + (tb + g * N + m0 + i) * 16);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float4 L = L4[p];
        const float o = fmaf(L.w, s3, fmaf(L.z, s2, fmaf(L.y, s1, fmaf(L.x, s0, r.t[i][p]))));
        const float d = o - r.old[i][p];
        e2 = fmaf(d, d, e2);
        ob[(i * 4 + p) * T] = o;
      }
    }
  }
  return e2;
}

// A block's tiles of one sweep with the loads of tile k+1 issued before tile k
// is computed (the input buffer is read-only within a sweep).
template <int T, int NP>
__device__ __forceinline__ float tiled_sweep_pf(int J, int N, int G, int cl, int gy, bool zero,
                                                const int32_t *__restrict__ type, const float *Linv, const float *Cin,
                                                const float *Mp, const float *w, const float *__restrict__ z,
                                                const float *__restrict__ Din, float *__restrict__ Dout, float *y_s,
                                                float *yr_s, float *s_s) {
  const int ntiles = (J + T - 1) / T;
  float e2 = 0.f;
  int tile = blockIdx.x;
  if (tile >= ntiles) return e2;
  TileRegs<NP> a, b;
  tiled_load<T, NP>(a, tile, J, N, G, cl, gy, zero, type, z, Din);
  for (;;) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles) tiled_load<T, NP>(b, nxt, J, N, G, cl, gy, zero, type, z, Din);
    e2 += tiled_compute<T, NP>(a, tile, N, G, cl, gy, Linv, Cin, Mp, w, Dout, y_s, yr_s, s_s);
    if (nxt >= ntiles) break;
    tile = nxt;
    a = b;
  }
  return e2;
}


template <int T, int NP>
__global__ void __launch_bounds__(256) k_mx_inner_tp(int J, int N, int G, int n_types, int stage,
                                                     const int32_t *__restrict__ type, const float *Linv_g,
                                                     const float *Cin_g, const float *Mp_g, const float *w_g,
                                                     const float *__restrict__ z, float *D0, float *D1, DevState *ds,
                                                     double *__restrict__ partials, unsigned *counter,
                                                     double *e_hist, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) float smr[];
  __shared__ double red[8];
  __shared__ bool s_last;
  const int P = N / NP, G4 = 4 * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (ds->done) return;  // uniform across the grid
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  float *y_s = smr;
  float *yr_s = y_s + (size_t)G * P * 4 * T;
  float *s_s = yr_s + (size_t)G4 * T;
  const float *Linv = Linv_g, *Cin = Cin_g, *Mp = Mp_g, *w = w_g;
  if (stage) {
    stage_tables(s_s + (size_t)G4 * T, n_types, N, G, tid, nthr, Linv, Cin, Mp, w);
    __syncthreads();
  }
  const int ntiles = (J + T - 1) / T;
  float e2 = 0.f;
  if (NP <= 4)
    e2 = tiled_sweep_pf<T, NP>(J, N, G, cl, gy, zero, type, Linv, Cin, Mp, w, z, Din, Dout, y_s, yr_s, s_s);
  else
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      e2 += tiled_tile<T, NP>(tile, J, N, G, cl, gy, zero, type, Linv, Cin, Mp, w, z, Din, Dout, y_s, yr_s, s_s);
  const double bs = block_reduce_fixed(e2, red, tid, nthr);
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

// ---------------------------------------------------------------- inner sweeps, multi-sweep
// Consecutive inner sweeps of the persistent tiled form in one cooperative
// launch (all blocks resident): after each sweep a grid barrier, then every
// block sums the per-block partials in the same fixed order, so all blocks
// reach the same e and take the same stop-rule and refinement decision on
// their copy of the device state.  The launch ends when the stop rule holds
// or a refinement is due (the graph's IF node then runs the FP64 refinement
// and the WHILE loop relaunches).  Partials are double-buffered by sweep
// parity: a block that starts the next sweep cannot overwrite values another
// block is still summing.  The barrier spin is bounded; a timeout records
// OCI_E_TIMEOUT and ends the step.

template <int T, int NP>
__global__ void __launch_bounds__(256) k_mx_inner_ms(int J, int N, int G, int n_types, int stage,
                                                     const int32_t *__restrict__ type, const float *Linv_g,
                                                     const float *Cin_g, const float *Mp_g, const float *w_g,
                                                     const float *__restrict__ z, float *D0, float *D1, DevState *ds,
                                                     double *__restrict__ partials, unsigned long long *gbar, double *e_hist,
                                                     cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  extern __shared__ __align__(16) float smr[];
  __shared__ double red[8];
  __shared__ DevState sd;
  __shared__ int s_ok;
  unsigned long long gep = 0;  // thread 0: the arrival count the next grid barrier waits for
  const int P = N / NP, G4 = 4 * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the grid
  float *y_s = smr;
  float *yr_s = y_s + (size_t)G * P * 4 * T;
  float *s_s = yr_s + (size_t)G4 * T;
  const float *Linv = Linv_g, *Cin = Cin_g, *Mp = Mp_g, *w = w_g;
  if (stage) {
    stage_tables(s_s + (size_t)G4 * T, n_types, N, G, tid, nthr, Linv, Cin, Mp, w);
    __syncthreads();
  }
  const int ntiles = (J + T - 1) / T;
  bool failed = false;
  for (int sw = 0;; sw++) {
    const bool zero = sd.refine || sd.blk_i == 0;
    const float *__restrict__ Din = sd.dcur ? D1 : D0;
    float *__restrict__ Dout = sd.dcur ? D0 : D1;
    float e2 = 0.f;
    if (NP <= 4)
      e2 = tiled_sweep_pf<T, NP>(J, N, G, cl, gy, zero, type, Linv, Cin, Mp, w, z, Din, Dout, y_s, yr_s, s_s);
    else
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        e2 += tiled_tile<T, NP>(tile, J, N, G, cl, gy, zero, type, Linv, Cin, Mp, w, z, Din, Dout, y_s, yr_s, s_s);
    const double bs = block_reduce_fixed(e2, red, tid, nthr);
    double *part = partials + (size_t)(sw & 1) * gridDim.x;
    if (tid == 0) {
      part[blockIdx.x] = bs;
      s_ok = grid_barrier_count(gbar, gep += gridDim.x, sd.spin);
    }
    __syncthreads();
    if (!s_ok) {
      failed = true;
      break;
    }
    const double tot = block_sum_fixed(part, gridDim.x, red);
    if (tid == 0) finish_mixed(&sd, blockIdx.x == 0 ? e_hist : nullptr, sqrt(tot), cond, 0);
    __syncthreads();
    if (sd.done || sd.refine || sw + 1 >= max_sweeps) break;  // uniform: every block holds the same state
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (failed) {
      sd.status = OCI_E_TIMEOUT;
      sd.done = 1;
      sd.refine = 0;
    }
    *ds = sd;
    if (use_cond) {
      if (sd.done) cudaGraphSetConditional(cond, 0);
      if (sd.cond_ref) cudaGraphSetConditional((cudaGraphConditionalHandle)sd.cond_ref, sd.refine);
    }
  }
}

template <int T, int NP>
static int ms_grid(const Handle &h, int P, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_ms<T, NP>, T * h.G * P, smem);
  const int ntiles = (h.J + T - 1) / T;
  const int grid = sms * per;
  return grid < ntiles ? grid : ntiles;
}

template <int T, int NP>
static void launch_ms(Handle &h, int P, size_t smem, bool stage, cudaGraphConditionalHandle cond, int use_cond,
                      int max_sweeps) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ms_grid<T, NP>(h, P, smem));
  cfg.blockDim = dim3(T, h.G * P);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  k_zero_gcount<<<1, 1, 0, h.stream>>>(reinterpret_cast<unsigned long long *>(h.gbar));
  cudaLaunchKernelEx(&cfg, k_mx_inner_ms<T, NP>, h.J, h.N, h.G, h.tt.n_types, (int)stage, (const int32_t *)h.type,
                     (const float *)h.tt.Linv32, (const float *)h.tt.Cin32, (const float *)h.tt.Mp32,
                     (const float *)h.w32, (const float *)h.z32, h.delta[0], h.delta[1], h.ds, h.partials, reinterpret_cast<unsigned long long *>(h.gbar),
                     h.e_hist, cond, use_cond, max_sweeps);
}

template <int T, int NP>
static int tp_grid(const Handle &h, int P, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_tp<T, NP>, T * h.G * P, smem);
  const int ntiles = (h.J + T - 1) / T;
  const int grid = sms * per;
  return grid < ntiles ? grid : ntiles;
}

// ---------------------------------------------------------------- inner sweep, tiled + bulk copies
// The persistent tiled sweep with each tile's operands brought into shared
// memory by the tensor memory accelerator: in the tile-major layout a tile's
// z and delta_in are each one contiguous chunk of 4NG*T floats, so one 1D bulk
// copy (cp.async.bulk, completing on an mbarrier) per array moves them.  Two
// stages: the copies of the block's next tile are in flight while the current
// tile is computed.  Only the upstream edge of a tile's first / last column is
// read from global memory (the adjacent tile).  Every wait is bounded: on a
// timeout the block records OCI_E_TIMEOUT, waits (bounded) for its copies still
// in flight and leaves.
constexpr long long kBulkSpin = 1 << 22;

__device__ __forceinline__ void bulk_load_1d(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  uint32_t ok = 0;
  for (long long k = 0; k < kBulkSpin && !ok; k++)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
  return ok != 0;
}

size_t mx_tb_smem(const Handle &h, int T, int P, bool stage) {
  const size_t chunk = (size_t)4 * h.N * h.G * T;
  return 4 * chunk * 4 + mx_tp_smem(h, T, P, stage) + 128;
}

template <int T, int NP>
__global__ void __launch_bounds__(256) k_mx_inner_tb(int J, int N, int G, int n_types, int stage,
                                                     const int32_t *__restrict__ type, const float *Linv_g,
                                                     const float *Cin_g, const float *Mp_g, const float *w_g,
                                                     const float *__restrict__ z, float *D0, float *D1, DevState *ds,
                                                     double *__restrict__ partials, unsigned *counter,
                                                     double *e_hist, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(128) unsigned char smb_[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ double red[8];
  __shared__ bool s_last;
  const int P = N / NP, G4 = 4 * G, R = 4 * N * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (ds->done) return;  // uniform across the grid
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  float *smb = (float *)(((uintptr_t)smb_ + 127) & ~(uintptr_t)127);
  const size_t chunk = (size_t)R * T;  // floats of one array in one tile
  const uint32_t cbytes = (uint32_t)(chunk * 4);
  const uint32_t tx = zero ? cbytes : 2 * cbytes;
  float *y_s = smb + 4 * chunk;  // stages: [st][z, delta][chunk]
  float *yr_s = y_s + (size_t)G * P * 4 * T;
  float *s_s = yr_s + (size_t)G4 * T;
  const float *Linv = Linv_g, *Cin = Cin_g, *Mp = Mp_g, *w = w_g;
  if (stage) {
    float *tab = s_s + (size_t)G4 * T;
    const size_t nL = (size_t)n_types * G * N * 16, nC = (size_t)n_types * G * N * 8;
    const size_t nM = (size_t)n_types * G4 * G4;
    float *sL = tab, *sC = sL + nL, *sM = sC + nC, *sw = sM + nM;
    for (size_t i = tid; i < nL; i += nthr) sL[i] = Linv_g[i];
    for (size_t i = tid; i < nC; i += nthr) sC[i] = Cin_g[i];
    for (size_t i = tid; i < nM; i += nthr) sM[i] = Mp_g[i];
    for (int i = tid; i < N; i += nthr) sw[i] = w_g[i];
    Linv = sL;
    Cin = sC;
    Mp = sM;
    w = sw;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const int ntiles = (J + T - 1) / T;
  auto issue = [&](int tile, int st) {  // thread 0
    const uint32_t bar = smem_addr(&mbar[st]);
    float *dst = smb + (size_t)st * 2 * chunk;
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
    bulk_load_1d(smem_addr(dst), z + (size_t)tile * chunk, cbytes, bar);
    if (!zero) bulk_load_1d(smem_addr(dst + chunk), Din + (size_t)tile * chunk, cbytes, bar);
  };
  const int N2 = N / 2;
  float e2 = 0.f;
  int it = 0;
  bool failed = false;
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int st = it & 1;
    // stage st^1 was last read before the y_s barrier of the previous tile
    if (tid == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, st ^ 1);
    const bool ok = mbar_wait_bounded(smem_addr(&mbar[st]), (uint32_t)((it >> 1) & 1));
    if (!__syncthreads_and(ok)) {  // the same decision in every thread
      failed = true;
      break;
    }
    const float *zs = smb + (size_t)st * 2 * chunk;
    const float *dsm = zs + chunk;
    const int j = tile * T + cl;
    const bool active = j < J;
    const int tau = active ? type[j] : 0;
    const size_t tb = (size_t)tau * G * N;
    const int row0 = (g * N + m0) * 4;
    float t[NP][4], old[NP][4];
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const int m = m0 + i;
        const int r = row0 + i * 4;
#pragma unroll
        for (int p = 0; p < 4; p++) {
          t[i][p] = zs[(r + p) * T + cl];
          old[i][p] = zero ? 0.f : dsm[(r + p) * T + cl];
        }
        float uk = 0.f, uh = 0.f;
        if (!zero) {
          if (m >= N2) {  // R corner of cell j-1
            if (cl > 0) {
              uk = dsm[(r + 1) * T + cl - 1];
              uh = dsm[(r + 3) * T + cl - 1];
            } else if (j > 0) {
              const float *prev = Din + ((size_t)(tile - 1) * R) * T + (T - 1);
              uk = prev[(size_t)(r + 1) * T];
              uh = prev[(size_t)(r + 3) * T];
            }
          } else {  // L corner of cell j+1
            if (j < J - 1) {
              if (cl < T - 1) {
                uk = dsm[(r + 0) * T + cl + 1];
                uh = dsm[(r + 2) * T + cl + 1];
              } else {
                const float *next = Din + ((size_t)(tile + 1) * R) * T;
                uk = next[(size_t)(r + 0) * T];
                uh = next[(size_t)(r + 2) * T];
              }
            }
          }
        }
        const float4 *C4 = reinterpret_cast<const float4 *>(Cin + (tb + g * N + m) * 8);
        const float4 ca = C4[0], cb = C4[1];
        t[i][0] = fmaf(ca.y, uh, fmaf(ca.x, uk, t[i][0]));
        t[i][1] = fmaf(ca.w, uh, fmaf(ca.z, uk, t[i][1]));
        t[i][2] = fmaf(cb.y, uh, fmaf(cb.x, uk, t[i][2]));
        t[i][3] = fmaf(cb.w, uh, fmaf(cb.z, uk, t[i][3]));
        const float wm = w[m];
        y0 = fmaf(wm, t[i][0], y0);
        y1 = fmaf(wm, t[i][1], y1);
        y2 = fmaf(wm, t[i][2], y2);
        y3 = fmaf(wm, t[i][3], y3);
      }
    }
    {
      float *ys = y_s + (size_t)(gy * 4) * T + cl;
      ys[0] = y0;
      ys[T] = y1;
      ys[2 * T] = y2;
      ys[3 * T] = y3;
    }
    __syncthreads();
    for (int q = ch; q < 4; q += P) {
      float v = y_s[(size_t)((g * P) * 4 + q) * T + cl];
      for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * T + cl];
      yr_s[(size_t)(g * 4 + q) * T + cl] = v;
    }
    __syncthreads();
    if (active)
      for (int q = ch; q < 4; q += P) {
        const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
        float v = 0.f;
        for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[(size_t)k * T + cl], v);
        s_s[(size_t)(g * 4 + q) * T + cl] = v;
      }
    __syncthreads();
    if (active) {
      const float s0 = s_s[(size_t)(g * 4 + 0) * T + cl], s1 = s_s[(size_t)(g * 4 + 1) * T + cl];
      const float s2 = s_s[(size_t)(g * 4 + 2) * T + cl], s3 = s_s[(size_t)(g * 4 + 3) * T + cl];
      float *ob = Dout + (size_t)tile * chunk + (size_t)row0 * T + cl;
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const float4 *L4 = reinterpret_cast<const float4 *>(Linv + (tb + g * N + m0 + i) * 16);
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const float4 L = L4[p];
          const float o = fmaf(L.w, s3, fmaf(L.z, s2, fmaf(L.y, s1, fmaf(L.x, s0, t[i][p]))));
          const float d = o - old[i][p];
          e2 = fmaf(d, d, e2);
          ob[(i * 4 + p) * T] = o;
        }
      }
    }
  }
  if (failed) {
    if (tid == 0) {  // let the copies still in flight land before the block's memory is released
      mbar_wait_bounded(smem_addr(&mbar[it & 1]), (uint32_t)((it >> 1) & 1));
      if (blockIdx.x + (it + 1) * gridDim.x < (unsigned)ntiles)
        mbar_wait_bounded(smem_addr(&mbar[(it + 1) & 1]), (uint32_t)(((it + 1) >> 1) & 1));
      atomicExch(&ds->status, OCI_E_TIMEOUT);
      ds->done = 1;
    }
    __syncthreads();
  }
  double v = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

template <int T, int NP>
static int tb_grid(const Handle &h, int P, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_tb<T, NP>, T * h.G * P, smem);
  const int ntiles = (h.J + T - 1) / T;
  const int grid = sms * per;
  return grid < ntiles ? grid : ntiles;
}

// ---------------------------------------------------------------- inner sweeps, red-black
// Red-black ordering of the mixed form: each inner sweep updates the even
// ("red") cells from their odd neighbours, then the odd ("black") cells from the
// new red values, in place on one correction buffer (two-colour block
// Gauss-Seidel on the same A and B).  The correction arrays are tile-major with
// each tile's columns ordered by colour, so a half sweep reads and writes
// contiguous half-tiles.  A grid barrier separates the colours (a black cell at
// a tile edge reads a red cell of the adjacent tile), so the kernel is always
// launched cooperatively: with max_sweeps = 1 outside the graph (one sweep per
// launch), and in the graph for consecutive sweeps until a refinement or the
// stop rule, like the Jacobi multi-sweep kernel.  On the first sweep after a
// refinement the buffer holds the previous block's correction: the red half
// reads no neighbours and both halves take their old values as zero.
template <int T, int NP>
__device__ __forceinline__ float rb_tile(int tile, int color, int J, int N, int G, int cl, int gy, bool zero,
                                         const int32_t *__restrict__ type, const float *Linv, const float *Cin,
                                         const float *Mp, const float *w, const float *__restrict__ z, float *D,
                                         float *y_s, float *yr_s, float *s_s) {
  constexpr int TH = T / 2;
  const int P = N / NP, G4 = 4 * G, R = 4 * N * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int N2 = N / 2;
  const int j = tile * T + 2 * cl + color;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const size_t tb = (size_t)tau * G * N;
  const int row0 = (g * N + m0) * 4;
  const size_t tbase = (size_t)tile * R * T;
  const size_t off = tbase + (size_t)row0 * T + color * TH + cl;
  // columns of the upstream cells j-1 (its R corner) and j+1 (its L corner)
  long long offL, offR;
  if (color == 0) {
    offL = cl > 0 ? (long long)(TH + cl - 1) : (long long)(T - 1) - (long long)R * T;  // black j-1
    offR = TH + cl;                                                                     // black j+1
  } else {
    offL = cl;                                                                      // red j-1
    offR = cl + 1 < TH ? (long long)(cl + 1) : (long long)R * T;                    // red j+1
  }
  const bool read_nb = !zero || color == 1;
  const float *zb = z + off;
  float *db = D + off;
  const float *nb = D + tbase + (size_t)row0 * T;  // + offL / offR + (i*4+p)*T
  float t[NP][4], old[NP][4];
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (active) {
    float uk[NP], uh[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        t[i][p] = zb[(i * 4 + p) * T];
        old[i][p] = zero ? 0.f : db[(i * 4 + p) * T];
      }
      uk[i] = 0.f;
      uh[i] = 0.f;
      if (read_nb) {
        if (m >= N2) {
          if (j > 0) {
            uk[i] = nb[offL + (i * 4 + 1) * T];
            uh[i] = nb[offL + (i * 4 + 3) * T];
          }
        } else if (j < J - 1) {
          uk[i] = nb[offR + (i * 4 + 0) * T];
          uh[i] = nb[offR + (i * 4 + 2) * T];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const float4 *C4 = reinterpret_cast<const float4 *>(Cin + (tb + g * N + m) * 8);
      const float4 ca = C4[0], cb = C4[1];
      t[i][0] = fmaf(ca.y, uh[i], fmaf(ca.x, uk[i], t[i][0]));
      t[i][1] = fmaf(ca.w, uh[i], fmaf(ca.z, uk[i], t[i][1]));
      t[i][2] = fmaf(cb.y, uh[i], fmaf(cb.x, uk[i], t[i][2]));
      t[i][3] = fmaf(cb.w, uh[i], fmaf(cb.z, uk[i], t[i][3]));
      const float wm = w[m];
      y0 = fmaf(wm, t[i][0], y0);
      y1 = fmaf(wm, t[i][1], y1);
      y2 = fmaf(wm, t[i][2], y2);
      y3 = fmaf(wm, t[i][3], y3);
    }
  }
  {
    float *ys = y_s + (size_t)(gy * 4) * TH + cl;
    ys[0] = y0;
    ys[TH] = y1;
    ys[2 * TH] = y2;
    ys[3 * TH] = y3;
  }
  __syncthreads();
  for (int q = ch; q < 4; q += P) {
    float v = y_s[(size_t)((g * P) * 4 + q) * TH + cl];
    for (int k = 1; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * TH + cl];
    yr_s[(size_t)(g * 4 + q) * TH + cl] = v;
  }
  __syncthreads();
  if (active)
    for (int q = ch; q < 4; q += P) {
      const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
      float v = 0.f;
      for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[(size_t)k * TH + cl], v);
      s_s[(size_t)(g * 4 + q) * TH + cl] = v;
    }
  __syncthreads();
  float e2 = 0.f;
  if (active) {
    const float s0 = s_s[(size_t)(g * 4 + 0) * TH + cl], s1 = s_s[(size_t)(g * 4 + 1) * TH + cl];
    const float s2 = s_s[(size_t)(g * 4 + 2) * TH + cl], s3 = s_s[(size_t)(g * 4 + 3) * TH + cl];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const float4 *L4 = reinterpret_cast<const float4 *>(Linv + (tb + g * N + m0 + i) * 16);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float4 L = L4[p];
        const float o = fmaf(L.w, s3, fmaf(L.z, s2, fmaf(L.y, s1, fmaf(L.x, s0, t[i][p]))));
        const float d = o - old[i][p];
        e2 = fmaf(d, d, e2);
        db[(i * 4 + p) * T] = o;
      }
    }
  }
  return e2;
}

template <int T, int NP>
__global__ void __launch_bounds__(256) k_mx_rb(int J, int N, int G, int n_types, int stage,
                                               const int32_t *__restrict__ type, const float *Linv_g,
                                               const float *Cin_g, const float *Mp_g, const float *w_g,
                                               const float *__restrict__ z, float *D, DevState *ds,
                                               double *__restrict__ partials, unsigned long long *gbar, double *e_hist,
                                               cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  extern __shared__ __align__(16) float smr[];
  __shared__ double red[8];
  __shared__ DevState sd;
  __shared__ int s_ok;
  unsigned long long gep = 0;  // thread 0: the arrival count the next grid barrier waits for
  constexpr int TH = T / 2;
  const int P = N / NP, G4 = 4 * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the grid
  float *y_s = smr;
  float *yr_s = y_s + (size_t)G * P * 4 * TH;
  float *s_s = yr_s + (size_t)G4 * TH;
  const float *Linv = Linv_g, *Cin = Cin_g, *Mp = Mp_g, *w = w_g;
  if (stage) {
    stage_tables(s_s + (size_t)G4 * TH, n_types, N, G, tid, nthr, Linv, Cin, Mp, w);
    __syncthreads();
  }
  const int ntiles = (J + T - 1) / T;
  bool failed = false;
  for (int sw = 0;; sw++) {
    const bool zero = sd.refine || sd.blk_i == 0;
    float e2 = 0.f;
    for (int color = 0; color < 2 && !failed; color++) {
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        e2 += rb_tile<T, NP>(tile, color, J, N, G, cl, gy, zero, type, Linv, Cin, Mp, w, z, D, y_s, yr_s, s_s);
      if (color == 0) {  // every red cell is written before any black cell reads it
        __syncthreads();
        if (tid == 0) s_ok = grid_barrier_count(gbar, gep += gridDim.x, sd.spin);
        __syncthreads();
        if (!s_ok) failed = true;
      }
    }
    if (failed) break;
    const double bs = block_reduce_fixed(e2, red, tid, nthr);
    double *part = partials + (size_t)(sw & 1) * gridDim.x;
    if (tid == 0) {
      part[blockIdx.x] = bs;
      s_ok = grid_barrier_count(gbar, gep += gridDim.x, sd.spin);
    }
    __syncthreads();
    if (!s_ok) {
      failed = true;
      break;
    }
    const double tot = block_sum_fixed(part, gridDim.x, red);
    if (tid == 0) finish_mixed(&sd, blockIdx.x == 0 ? e_hist : nullptr, sqrt(tot), cond, 0);
    __syncthreads();
    if (sd.done || sd.refine || sw + 1 >= max_sweeps) break;  // uniform
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (failed) {
      sd.status = OCI_E_TIMEOUT;
      sd.done = 1;
      sd.refine = 0;
    }
    *ds = sd;
    if (use_cond) {
      if (sd.done) cudaGraphSetConditional(cond, 0);
      if (sd.cond_ref) cudaGraphSetConditional((cudaGraphConditionalHandle)sd.cond_ref, sd.refine);
    }
  }
}

template <int T, int NP>
static void launch_rb(Handle &h, int P, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
  const size_t smem = mx_reg_smem(h.G, T / 2, P) + (stage ? mx_tables_floats(h) * 4 + 16 : 0);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_rb<T, NP>, (T / 2) * h.G * P, smem);
  const int ntiles = (h.J + T - 1) / T;
  int grid = sms * per;
  if (grid > ntiles) grid = ntiles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T / 2, h.G * P);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // blocks wait on one another (grid barriers)
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  k_zero_gcount<<<1, 1, 0, h.stream>>>(reinterpret_cast<unsigned long long *>(h.gbar));
  cudaLaunchKernelEx(&cfg, k_mx_rb<T, NP>, h.J, h.N, h.G, h.tt.n_types, (int)stage, (const int32_t *)h.type,
                     (const float *)h.tt.Linv32, (const float *)h.tt.Cin32, (const float *)h.tt.Mp32,
                     (const float *)h.w32, (const float *)h.z32, h.delta[0], h.ds, h.partials, reinterpret_cast<unsigned long long *>(h.gbar), h.e_hist,
                     cond, use_cond, max_sweeps);
}

// ---------------------------------------------------------------- inner sweep, TMA-staged
// The same FP32 inner sweep with the tile's operands brought in by the tensor
// memory accelerator: per tile of kTmaCells cells, one 2D bulk tensor copy
// moves z[0:R][j0:j0+64] and one moves delta_in[0:R][j0-4:j0+68] (the halo
// columns j0-1 and j0+64 are inside; x starts on a 16-byte boundary; columns
// outside the array read as zero, which is the correction's zero inflow at the
// slab ends) into shared memory, completing on an mbarrier.  A persistent CTA
// double-buffers the stages: the copy of its next tile is in flight while the
// current one is computed.  R = 4NG <= 256 (one box per operand).
constexpr int kTmaCells = 64;
constexpr int kTmaHalo = 4;                    // columns each side of the delta box
constexpr int kTmaDW = kTmaCells + 2 * kTmaHalo;  // delta box width
constexpr long long kTmaSpin = 1 << 22;


__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__global__ void __launch_bounds__(256) k_mx_inner_tma(const __grid_constant__ CUtensorMap tmZ,
                                                      const __grid_constant__ CUtensorMap tmD0,
                                                      const __grid_constant__ CUtensorMap tmD1, int J, int Jp, int N,
                                                      int G, int P, const int32_t *__restrict__ type,
                                                      const float *__restrict__ Linv, const float *__restrict__ Cin,
                                                      const float *__restrict__ Mp, const float *__restrict__ w,
                                                      float *D0, float *D1, DevState *ds,
                                                      double *__restrict__ partials, unsigned *counter,
                                                      double *e_hist, cudaGraphConditionalHandle cond,
                                                      int use_cond) {
  extern __shared__ __align__(1024) unsigned char smraw_[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ double red[32];
  __shared__ bool s_last;
  // stage buffers start on a 1024-byte boundary (the launch reserves 1 KiB extra)
  unsigned char *smraw = (unsigned char *)(((uintptr_t)smraw_ + 1023) & ~(uintptr_t)1023);
  const int R = 4 * N * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P;
  const int NP = N / P, m0 = ch * NP;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const CUtensorMap *tmDin = dcur ? &tmD1 : &tmD0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  // stage layout: z [R][64] then delta [R][72], each stage 1024-aligned
  const size_t zbytes = (size_t)R * kTmaCells * 4, dbytes = (size_t)R * kTmaDW * 4;
  const size_t stage_bytes = (zbytes + dbytes + 1023) / 1024 * 1024;
  float *y_s = (float *)(smraw + 2 * stage_bytes);  // [G*P*4][64]
  const uint32_t tx = (uint32_t)(zbytes + (zero ? 0 : dbytes));
  const int ntiles = (J + kTmaCells - 1) / kTmaCells;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  auto issue = [&](int tile, int st) {
    const uint32_t bar = smem_addr(&mbar[st]);
    unsigned char *base = smraw + st * stage_bytes;
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
    tma_load_2d(smem_addr(base), &tmZ, tile * kTmaCells, 0, bar);
    if (!zero) tma_load_2d(smem_addr(base + zbytes), tmDin, tile * kTmaCells - kTmaHalo, 0, bar);
  };
  const int N2 = N / 2;
  const int G4 = 4 * G;
  float e2 = 0.f;
  int it = 0;
  bool failed = false;
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int st = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    if (tid == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, st ^ 1);
    uint32_t ok = 0;
    for (long long k = 0; k < kTmaSpin && !ok; k++) {
      asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                   : "=r"(ok)
                   : "r"(smem_addr(&mbar[st])), "r"(parity)
                   : "memory");
    }
    if (!__syncthreads_and(ok)) {  // the same decision in every thread
      failed = true;
      break;
    }
    const float *zs = (const float *)(smraw + st * stage_bytes);
    const float *ds_ = (const float *)(smraw + st * stage_bytes + zbytes);
    const int j = tile * kTmaCells + cl;
    const bool active = j < J;
    const int tau = active ? type[j] : 0;
    const size_t tb = (size_t)tau * G * N;
    auto dval = [&](int r, int col) -> float { return zero ? 0.f : ds_[r * kTmaDW + col]; };
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
    if (active) {
      for (int m = m0; m < m0 + NP; m++) {
        const int gm = g * N + m;
        float uk, uh;
        if (m >= N2) {  // upstream R corner of cell j-1 (zero beyond the slab end)
          uk = dval(gm * 4 + 1, cl + kTmaHalo - 1);
          uh = dval(gm * 4 + 3, cl + kTmaHalo - 1);
        } else {  // upstream L corner of cell j+1
          uk = (j < J - 1) ? dval(gm * 4 + 0, cl + kTmaHalo + 1) : 0.f;
          uh = (j < J - 1) ? dval(gm * 4 + 2, cl + kTmaHalo + 1) : 0.f;
        }
        const float *C = Cin + (tb + gm) * 8;
        const float wm = w[m];
        y0 = fmaf(wm, fmaf(C[1], uh, fmaf(C[0], uk, zs[(gm * 4 + 0) * kTmaCells + cl])), y0);
        y1 = fmaf(wm, fmaf(C[3], uh, fmaf(C[2], uk, zs[(gm * 4 + 1) * kTmaCells + cl])), y1);
        y2 = fmaf(wm, fmaf(C[5], uh, fmaf(C[4], uk, zs[(gm * 4 + 2) * kTmaCells + cl])), y2);
        y3 = fmaf(wm, fmaf(C[7], uh, fmaf(C[6], uk, zs[(gm * 4 + 3) * kTmaCells + cl])), y3);
      }
    }
    y_s[(gy * 4 + 0) * kTmaCells + cl] = y0;
    y_s[(gy * 4 + 1) * kTmaCells + cl] = y1;
    y_s[(gy * 4 + 2) * kTmaCells + cl] = y2;
    y_s[(gy * 4 + 3) * kTmaCells + cl] = y3;
    __syncthreads();
    if (active) {
      const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int k = 0; k < G4; k++) {
        const int gp = k >> 2, q = k & 3;
        float yk = 0.f;
        for (int c = 0; c < P; c++) yk += y_s[((gp * P + c) * 4 + q) * kTmaCells + cl];
        s0 = fmaf(M[k], yk, s0);
        s1 = fmaf(M[G4 + k], yk, s1);
        s2 = fmaf(M[2 * G4 + k], yk, s2);
        s3 = fmaf(M[3 * G4 + k], yk, s3);
      }
      for (int m = m0; m < m0 + NP; m++) {
        const int gm = g * N + m;
        float uk, uh;
        if (m >= N2) {
          uk = dval(gm * 4 + 1, cl + kTmaHalo - 1);
          uh = dval(gm * 4 + 3, cl + kTmaHalo - 1);
        } else {
          uk = (j < J - 1) ? dval(gm * 4 + 0, cl + kTmaHalo + 1) : 0.f;
          uh = (j < J - 1) ? dval(gm * 4 + 2, cl + kTmaHalo + 1) : 0.f;
        }
        const float *C = Cin + (tb + gm) * 8;
        const float *L = Linv + (tb + gm) * 16;
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const float t = fmaf(C[p * 2 + 1], uh, fmaf(C[p * 2 + 0], uk, zs[(gm * 4 + p) * kTmaCells + cl]));
          const float o = fmaf(L[p * 4 + 3], s3, fmaf(L[p * 4 + 2], s2, fmaf(L[p * 4 + 1], s1, fmaf(L[p * 4 + 0], s0, t))));
          const float d = o - dval(gm * 4 + p, cl + kTmaHalo);
          e2 = fmaf(d, d, e2);
          Dout[(size_t)(gm * 4 + p) * Jp + j] = o;
        }
      }
    }
    __syncthreads();  // stage st and y_s are free for the next tile
  }
  if (failed && tid == 0) {
    atomicExch(&ds->status, OCI_E_TIMEOUT);
    ds->done = 1;
  }
  double v = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

size_t mx_tma_smem(const Handle &h, int P) {
  const int R = 4 * h.N * h.G;
  const size_t zbytes = (size_t)R * kTmaCells * 4, dbytes = (size_t)R * kTmaDW * 4;
  const size_t stage_bytes = (zbytes + dbytes + 1023) / 1024 * 1024;
  return 2 * stage_bytes + (size_t)h.G * P * 4 * kTmaCells * 4 + 1024;
}

const void *k_mx_inner_tma_ptr() { return (const void *)k_mx_inner_tma; }

// Encode the three tensor maps (z and the two delta buffers, [R rows][Jp cols] FP32).
int mx_tma_setup(Handle &h) {
  const int R = 4 * h.N * h.G;
  if (R > 256) return OCI_OK;  // one box per operand only
  typedef CUresult (*Encode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Encode enc = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !enc) return OCI_OK;  // no TMA path: keep the plain kernel
  const cuuint64_t dims[2] = {(cuuint64_t)h.Jp, (cuuint64_t)R};
  const cuuint64_t strides[1] = {(cuuint64_t)h.Jp * 4};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t boxz[2] = {(cuuint32_t)kTmaCells, (cuuint32_t)R};
  const cuuint32_t boxd[2] = {(cuuint32_t)kTmaDW, (cuuint32_t)R};
  CUresult r1 = enc(&h.tm_z, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.z32, dims, strides, boxz, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(&h.tm_d[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.delta[0], dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r3 = enc(&h.tm_d[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.delta[1], dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS || r3 != CUDA_SUCCESS) return OCI_OK;
  e = cudaFuncSetAttribute(k_mx_inner_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mx_inner_tma)");
  h.tma_ok = true;
  return OCI_OK;
}

// ---------------------------------------------------------------- outer (FP64)
// mode 0: residual of Psi[cur] (start of a step, correction zero)
// mode 1: if ds->refine: Psi[cur^1] = Psi[cur] + delta[dcur]; unless the step is
//         done, residual of Psi[cur^1]
// mode 2: if ds->blk_i > 0: Psi[cur^1] = Psi[cur] + delta[dcur] (apply only)
// The residual r = c + s + inflow - L_c Psi (Eqs. oci, Aj, rhs_sg, scatter) is
// formed in FP64 and z = Linv r (FP32) is stored for the inner sweeps.
// The kernel is bound by the FP64 pipe, so with hwcvt = 0 the conversions
// between the FP32 correction / residual and FP64 run on the integer pipe
// (oci_cvt.cuh, exact) and, in mode 1, an upstream neighbour inside the tile
// is read back from Psi[cur^1] (written before the block barrier) instead of
// adding its correction again; hwcvt = 1 keeps the compiler's conversions and
// the recomputation.  Both give the same bits.
__global__ void __launch_bounds__(256) k_mx_outer(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                                  const double *__restrict__ Lco, const double *__restrict__ Kap,
                                                  const float *__restrict__ Linv32, const double *__restrict__ w,
                                                  const double *__restrict__ mu, const double *__restrict__ inc,
                                                  const double *__restrict__ cvec, double *Psi0, double *Psi1,
                                                  const float *D0, const float *D1, const DevState *__restrict__ ds,
                                                  int mode, int store_r, float *__restrict__ z32, int tsh,
                                                  int hwcvt) {
  extern __shared__ double smd[];
  const int CB = blockDim.x;
  const int R = 4 * N * G;
  const int cl = threadIdx.x, g = threadIdx.y;
  if (mode == 1 && !ds->refine) return;  // the common case: a small grid exits at once
  if (mode == 2 && ds->blk_i == 0) return;
  const bool apply = mode != 0;
  const bool resid = mode == 0 || (mode == 1 && !ds->done);
  const int cur = ds->cur;
  const double *__restrict__ Pin = cur ? Psi1 : Psi0;
  double *__restrict__ Pout = cur ? Psi0 : Psi1;
  const float *__restrict__ Dl = ds->dcur ? D1 : D0;
  const int N2 = N / 2;
  const int ntiles = (J + CB - 1) / CB;
  const bool reuse = apply && !hwcvt;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * CB + cl;
    const bool active = j < J;
    const int tau = active ? type[j] : 0;
    double ph[4] = {0.0, 0.0, 0.0, 0.0};
    if (active) {
      for (int m = 0; m < N; m++) {
        const int gm = g * N + m;
        const size_t base = (size_t)gm * 4 * Jp + j;
        const double wm = w[m];
#pragma unroll
        for (int p = 0; p < 4; p++) {
          double v = Pin[base + (size_t)p * Jp];
          if (apply) {
            v += cvt_f2d(hwcvt, Dl[fidx(tsh, R, Jp, gm * 4 + p, j)]);
            Pout[base + (size_t)p * Jp] = v;
          }
          ph[p] = fma(wm, v, ph[p]);
        }
      }
    }
    if (!resid) continue;  // uniform
    double *ph_s = smd;    // [G*4][CB]
    __syncthreads();       // previous tile's readers are done
#pragma unroll
    for (int p = 0; p < 4; p++) ph_s[(size_t)(g * 4 + p) * CB + cl] = ph[p];
    __syncthreads();
    if (!active) continue;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int gp = 0; gp < G; gp++) {
      const double k = Kap[((size_t)tau * G + gp) * G + g];
#pragma unroll
      for (int p = 0; p < 4; p++) s[p] = fma(k, ph_s[(size_t)(gp * 4 + p) * CB + cl], s[p]);
    }
    const double *P = apply ? Pout : Pin;  // Pout: written by this block before the barrier
    for (int m = 0; m < N; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const double v0 = P[base], v1 = P[base + (size_t)Jp], v2 = P[base + 2 * (size_t)Jp],
                   v3 = P[base + 3 * (size_t)Jp];
      const double *L = Lco + ((size_t)tau * G * N + gm) * 5;  // a, mu/2, alpha/2, alpha, alpha+a
      const double a = L[0], hm = L[1], ha = L[2], al = L[3], aa = L[4];
      double r0 = cvec[base] + s[0];
      double r1 = cvec[base + (size_t)Jp] + s[1];
      double r2 = cvec[base + 2 * (size_t)Jp] + s[2];
      double r3 = cvec[base + 3 * (size_t)Jp] + s[3];
      if (m >= N2) {  // mu > 0: upstream R corner of cell j-1 into rows 0, 2
        double uk, uh;
        if (j > 0) {
          const size_t nb = base - 1;
          if (reuse && cl > 0) {
            uk = Pout[nb + (size_t)Jp];
            uh = Pout[nb + 3 * (size_t)Jp];
          } else {
            uk = Pin[nb + (size_t)Jp];
            uh = Pin[nb + 3 * (size_t)Jp];
            if (apply) {
              uk += cvt_f2d(hwcvt, Dl[fidx(tsh, R, Jp, gm * 4 + 1, j - 1)]);
              uh += cvt_f2d(hwcvt, Dl[fidx(tsh, R, Jp, gm * 4 + 3, j - 1)]);
            }
          }
        } else {
          uk = inc[gm * 2 + 0];
          uh = inc[gm * 2 + 1];
        }
        r0 = fma(mu[m], uk, r0);
        r2 = fma(mu[m], uh, r2);
      } else {  // mu < 0: upstream L corner of cell j+1 into rows 1, 3
        double uk, uh;
        if (j < J - 1) {
          const size_t nb = base + 1;
          if (reuse && cl < CB - 1) {
            uk = Pout[nb];
            uh = Pout[nb + 2 * (size_t)Jp];
          } else {
            uk = Pin[nb];
            uh = Pin[nb + 2 * (size_t)Jp];
            if (apply) {
              uk += cvt_f2d(hwcvt, Dl[fidx(tsh, R, Jp, gm * 4 + 0, j + 1)]);
              uh += cvt_f2d(hwcvt, Dl[fidx(tsh, R, Jp, gm * 4 + 2, j + 1)]);
            }
          }
        } else {
          uk = inc[(G * N + gm) * 2 + 0];
          uh = inc[(G * N + gm) * 2 + 1];
        }
        r1 = fma(-mu[m], uk, r1);
        r3 = fma(-mu[m], uh, r3);
      }
      // r -= L_c Psi  (rows of Eq. Aj)
      r0 = fma(-a, v0, fma(-hm, v1, fma(-ha, v2, r0)));
      r1 = fma(hm, v0, fma(-a, v1, fma(-ha, v3, r1)));
      r2 = fma(al, v0, fma(-aa, v2, fma(-hm, v3, r2)));
      r3 = fma(al, v1, fma(hm, v2, fma(-aa, v3, r3)));
      const float f0 = cvt_d2f(hwcvt, r0), f1 = cvt_d2f(hwcvt, r1), f2 = cvt_d2f(hwcvt, r2), f3 = cvt_d2f(hwcvt, r3);
      if (store_r) {  // the tensor-core inner sweep applies the dense inverse to r itself
        z32[fidx(tsh, R, Jp, gm * 4 + 0, j)] = f0;
        z32[fidx(tsh, R, Jp, gm * 4 + 1, j)] = f1;
        z32[fidx(tsh, R, Jp, gm * 4 + 2, j)] = f2;
        z32[fidx(tsh, R, Jp, gm * 4 + 3, j)] = f3;
        continue;
      }
      const float *Li = Linv32 + ((size_t)tau * G * N + gm) * 16;
#pragma unroll
      for (int p = 0; p < 4; p++)
        z32[fidx(tsh, R, Jp, gm * 4 + p, j)] = fmaf(Li[p * 4 + 3], f3, fmaf(Li[p * 4 + 2], f2, fmaf(Li[p * 4 + 1], f1, Li[p * 4 + 0] * f0)));
    }
  }
}

// ---------------------------------------------------------------- control
__global__ void __launch_bounds__(kFinalizeThreads) k_mx_finalize(const double *__restrict__ partials, int n,
                                                                    DevState *ds, double *e_hist,
                                                                    cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double red[32];
  if (ds->done) {
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double tot = block_sum_fixed(partials, n, red);
  if (threadIdx.x == 0) finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
}

// kind 0: settle a pending refinement (flip Psi, zero correction)
// kind 1: after an apply-only outer kernel (mode 2), flip Psi
__global__ void k_mx_settle(DevState *ds, int kind) {
  if (kind == 0) {
    if (ds->refine) {
      ds->cur ^= 1;
      ds->refine = 0;
      ds->blk_i = 0;
    }
  } else if (ds->blk_i > 0) {
    ds->cur ^= 1;
    ds->blk_i = 0;
  }
}

void mx_shape(const Handle &h, int &cb, int &P) {
  cb = h.mx_kind == kMxTma ? kTmaCells : h.mx_cb;
  P = h.mx_P;
  if (cb > 0) return;
  P = 1;
  cb = 128;
  while (cb > 1 && ((size_t)cb * h.G > 256 || sweep_smem(h.N, h.G, cb, 1, 4) > 96 * 1024)) cb /= 2;
}

int tc_partials(const Handle &h);
int mx_partials(const Handle &h) {
  if (h.precision != OCI_FP32_IR) return tc_partials(h);
  if (h.mx_kind == kMxTma) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_tma, kTmaCells * h.G * h.mx_P,
                                                  mx_tma_smem(h, h.mx_P));
    const int ntiles = (h.J + kTmaCells - 1) / kTmaCells;
    const int grid = sms * per;
    return grid < ntiles ? grid : ntiles;
  }
  int cb, P;
  mx_shape(h, cb, P);
  const int ntiles = (h.J + cb - 1) / cb;
  // two sweeps x two parities per block
  return (h.mx_kind == kMxTiled2 || h.mx_kind == kMxTiled2Occ || h.mx_kind == kMxRB2 || h.mx_kind == kMxWarp2)
             ? 4 * ntiles
             : ntiles;
}

// One inner sweep including its norm reduction, stop rule and refinement
// decision (fused into the last block).
void launch_mx_inner(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  if (h.mx_kind == kMxRB2) {  // cooperative; in the graph passes of two red-black sweeps until an event
    const int ms = h.mx_tune_sweeps > 0 ? h.mx_tune_sweeps : (use_cond && h.mx_multi) ? (1 << 30) : 1;
    launch_rb2_any(h, cond, use_cond, ms);
    return;
  }
  if (h.mx_kind == kMxRB) {  // always cooperative; one sweep per launch outside the graph
    const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
    const int ms = h.mx_tune_sweeps > 0 ? h.mx_tune_sweeps : use_cond ? (1 << 30) : 1;
    if (T == 32) {
      if (np == 2) launch_rb<32, 2>(h, P, cond, use_cond, ms);
      else if (np == 4) launch_rb<32, 4>(h, P, cond, use_cond, ms);
      else launch_rb<32, 8>(h, P, cond, use_cond, ms);
    } else {
      if (np == 2) launch_rb<64, 2>(h, P, cond, use_cond, ms);
      else if (np == 4) launch_rb<64, 4>(h, P, cond, use_cond, ms);
      else launch_rb<64, 8>(h, P, cond, use_cond, ms);
    }
    return;
  }
  if (h.mx_kind == kMxTiledB) {
    const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
    const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
    const size_t smem = mx_tb_smem(h, T, P, stage);
    const dim3 block(T, h.G * P);
#define OCI_MX_TB(TT, NP)                                                                                        \
  k_mx_inner_tb<TT, NP><<<tb_grid<TT, NP>(h, P, smem), block, smem, h.stream>>>(                                 \
      h.J, h.N, h.G, h.tt.n_types, stage, h.type, h.tt.Linv32, h.tt.Cin32, h.tt.Mp32, h.w32, h.z32, h.delta[0], \
      h.delta[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond)
    if (T == 32) {
      if (np == 2) OCI_MX_TB(32, 2);
      else if (np == 4) OCI_MX_TB(32, 4);
      else OCI_MX_TB(32, 8);
    } else {
      if (np == 2) OCI_MX_TB(64, 2);
      else if (np == 4) OCI_MX_TB(64, 4);
      else OCI_MX_TB(64, 8);
    }
#undef OCI_MX_TB
    return;
  }
  if (h.mx_kind == kMxWarp2) {  // cooperative; in the graph passes of two sweeps
    const int ms = h.mx_tune_sweeps > 0 ? h.mx_tune_sweeps : (use_cond && h.mx_multi) ? (1 << 30) : 1;
    launch_w2_any(h, cond, use_cond, ms);
    return;
  }
  if (h.mx_kind == kMxTiled2 || h.mx_kind == kMxTiled2Occ) {  // cooperative; in the graph passes of two sweeps
    const int ms = h.mx_tune_sweeps > 0 ? h.mx_tune_sweeps : (use_cond && h.mx_multi) ? (1 << 30) : 1;
    launch_ms2_any(h, cond, use_cond, ms);
    return;
  }
  if (h.mx_kind == kMxTiledP && ((use_cond && h.mx_multi) || h.mx_tune_sweeps > 0)) {
    // in the graph (or when the autotuner times it): several sweeps per cooperative launch
    const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
    const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
    const size_t smem = mx_tp_smem(h, T, P, stage);
    const int ms = use_cond ? (1 << 30) : h.mx_tune_sweeps;
#define OCI_MS(TT, NP) launch_ms<TT, NP>(h, P, smem, stage, cond, use_cond, ms)
    if (T == 16) {
      OCI_MS(16, 8);
    } else if (T == 128) {
      OCI_MS(128, 8);
    } else if (T == 32) {
      if (np == 2) OCI_MS(32, 2);
      else if (np == 4) OCI_MS(32, 4);
      else OCI_MS(32, 8);
    } else {
      if (np == 2) OCI_MS(64, 2);
      else if (np == 4) OCI_MS(64, 4);
      else OCI_MS(64, 8);
    }
#undef OCI_MS
    return;
  }
  if (h.mx_kind == kMxTiledP) {
    const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
    const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
    const size_t smem = mx_tp_smem(h, T, P, stage);
    const dim3 block(T, h.G * P);
#define OCI_MX_TP(TT, NP)                                                                                        \
  k_mx_inner_tp<TT, NP><<<tp_grid<TT, NP>(h, P, smem), block, smem, h.stream>>>(                                 \
      h.J, h.N, h.G, h.tt.n_types, stage, h.type, h.tt.Linv32, h.tt.Cin32, h.tt.Mp32, h.w32, h.z32, h.delta[0], \
      h.delta[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond)
    if (T == 16) {
      OCI_MX_TP(16, 8);
    } else if (T == 128) {
      OCI_MX_TP(128, 8);
    } else if (T == 32) {
      if (np == 2) OCI_MX_TP(32, 2);
      else if (np == 4) OCI_MX_TP(32, 4);
      else OCI_MX_TP(32, 8);
    } else {
      if (np == 2) OCI_MX_TP(64, 2);
      else if (np == 4) OCI_MX_TP(64, 4);
      else OCI_MX_TP(64, 8);
    }
#undef OCI_MX_TP
    return;
  }
  if (h.mx_kind == kMxTiled) {
    const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
    const dim3 block(T, h.G * P), grid((h.J + T - 1) / T);
    const size_t smem = mx_tiled_smem(h.G, T, P);
#define OCI_MX_TILED(TT, NP)                                                                                     \
  k_mx_inner_tiled<TT, NP><<<grid, block, smem, h.stream>>>(h.J, h.N, h.G, h.type, h.tt.Linv32, h.tt.Cin32,      \
                                                            h.tt.Mp32, h.w32, h.z32, h.delta[0], h.delta[1], h.ds, \
                                                            h.partials, h.counter, h.e_hist, cond, use_cond)
    if (T == 32) {
      if (np == 2) OCI_MX_TILED(32, 2);
      else if (np == 4) OCI_MX_TILED(32, 4);
      else OCI_MX_TILED(32, 8);
    } else {
      if (np == 2) OCI_MX_TILED(64, 2);
      else if (np == 4) OCI_MX_TILED(64, 4);
      else OCI_MX_TILED(64, 8);
    }
#undef OCI_MX_TILED
    return;
  }
  if (h.mx_kind == kMxReg) {
    const int cb = h.mx_cb, P = h.mx_P, np = h.N / P;
    const dim3 block(cb, h.G * P), grid((h.J + cb - 1) / cb);
    const size_t smem = mx_reg_smem(h.G, cb, P);
#define OCI_MX_REG(NP)                                                                                        \
  k_mx_inner_reg<NP><<<grid, block, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Linv32, h.tt.Cin32,    \
                                                      h.tt.Mp32, h.w32, h.z32, h.delta[0], h.delta[1], h.ds, \
                                                      h.partials, h.counter, h.e_hist, cond, use_cond)
    if (np == 2) OCI_MX_REG(2);
    else if (np == 4) OCI_MX_REG(4);
    else OCI_MX_REG(8);
#undef OCI_MX_REG
    return;
  }
  if (h.mx_kind == kMxTma) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int P = h.mx_P;
    const size_t smem = mx_tma_smem(h, P);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_tma, kTmaCells * h.G * P, smem);
    const int ntiles = (h.J + kTmaCells - 1) / kTmaCells;
    int grid = sms * per;
    if (grid > ntiles) grid = ntiles;
    k_mx_inner_tma<<<grid, dim3(kTmaCells, h.G * P), smem, h.stream>>>(
        h.tm_z, h.tm_d[0], h.tm_d[1], h.J, h.Jp, h.N, h.G, P, h.type, h.tt.Linv32, h.tt.Cin32, h.tt.Mp32, h.w32,
        h.delta[0], h.delta[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond);
    return;
  }
  int cb, P;
  mx_shape(h, cb, P);
  dim3 block(cb, h.G * P);
  k_mx_inner<<<(h.J + cb - 1) / cb, block, sweep_smem(h.N, h.G, cb, P, 4), h.stream>>>(
      h.J, h.Jp, h.N, h.G, P, h.type, h.tt.Linv32, h.tt.Cin32, h.tt.Mp32, h.w32, h.z32, h.delta[0], h.delta[1], h.ds,
      h.partials, h.counter, h.e_hist, cond, use_cond);
}

void launch_mx_outer(Handle &h, int mode) {
  int cb = 128;
  while (cb > 1 && cb * h.G > 256) cb /= 2;
  dim3 block(cb, h.G);
  const size_t smem = (size_t)cb * h.G * 4 * sizeof(double);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (h.J + cb - 1) / cb;
  const int grid = ntiles < 4 * sms ? ntiles : 4 * sms;  // grid-stride over tiles
  k_mx_outer<<<grid, block, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Lco, h.tt.Kap,
                                                             h.tt.Linv32, h.w, h.mu, h.inc, h.tc, h.Psi[0], h.Psi[1],
                                                             h.delta[0], h.delta[1], h.ds, mode,
                                                             h.precision != OCI_FP32_IR, h.z32, mx_tile_shift(h),
                                                             h.mx_hwcvt);
}

void launch_mx_finalize(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  k_mx_finalize<<<1, kFinalizeThreads, 0, h.stream>>>(h.partials, mx_partials(h), h.ds, h.e_hist, cond, use_cond);
}

void launch_mx_settle(Handle &h, int kind) { k_mx_settle<<<1, 1, 0, h.stream>>>(h.ds, kind); }

const void *k_mx_inner_ptr() { return (const void *)k_mx_inner; }

// Dynamic shared memory limits of the FP32 inner kernels above 48 KB (set once at setup).
int mx_set_attributes() {
  const void *ks[] = {(const void *)k_mx_inner,          (const void *)k_mx_inner_tp<16, 8>,
                      (const void *)k_mx_inner_ms<16, 8>, (const void *)k_mx_inner_tp<128, 8>,
                      (const void *)k_mx_inner_ms<128, 8>, (const void *)k_mx_inner_tp<32, 2>,
                      (const void *)k_mx_inner_tp<32, 4>, (const void *)k_mx_inner_tp<32, 8>,
                      (const void *)k_mx_inner_tp<64, 2>, (const void *)k_mx_inner_tp<64, 4>,
                      (const void *)k_mx_inner_tp<64, 8>, (const void *)k_mx_inner_tb<32, 2>,
                      (const void *)k_mx_inner_tb<32, 4>, (const void *)k_mx_inner_tb<32, 8>,
                      (const void *)k_mx_inner_tb<64, 2>, (const void *)k_mx_inner_tb<64, 4>,
                      (const void *)k_mx_inner_tb<64, 8>, (const void *)k_mx_inner_ms<32, 2>,
                      (const void *)k_mx_inner_ms<32, 4>, (const void *)k_mx_inner_ms<32, 8>,
                      (const void *)k_mx_inner_ms<64, 2>, (const void *)k_mx_inner_ms<64, 4>,
                      (const void *)k_mx_inner_ms<64, 8>, (const void *)k_mx_rb<32, 2>,
                      (const void *)k_mx_rb<32, 4>, (const void *)k_mx_rb<32, 8>,
                      (const void *)k_mx_rb<64, 2>, (const void *)k_mx_rb<64, 4>,
                      (const void *)k_mx_rb<64, 8>};
  for (const void *k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(FP32 inner sweep)");
  }
  return mx_two_set_attributes();
}

}  // namespace oci
