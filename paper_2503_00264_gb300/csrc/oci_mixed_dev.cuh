// oci_mixed_dev.cuh -- device helpers shared by the FP32 inner-sweep kernels
// of the mixed form (oci_mixed.cu, oci_mixed_two.cu, oci_mixed_rb2.cu).
#pragma once
#include <stdint.h>

#include "oci_device.cuh"

namespace oci {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Per-type tables into shared memory (16-byte aligned sections); the pointers
// are redirected to the copies.  All threads; no barrier.
__device__ __forceinline__ void stage_tables(float *tab, int n_types, int N, int G, int tid, int nthr,
                                             const float *&Linv, const float *&Cin, const float *&Mp,
                                             const float *&w) {
  const int G4 = 4 * G;
  const size_t nL = (size_t)n_types * G * N * 16, nC = (size_t)n_types * G * N * 8;
  const size_t nM = (size_t)n_types * G4 * G4;
  float *sL = tab, *sC = sL + nL, *sM = sC + nC, *sw = sM + nM;
  for (size_t i = tid; i < nL; i += nthr) sL[i] = Linv[i];
  for (size_t i = tid; i < nC; i += nthr) sC[i] = Cin[i];
  for (size_t i = tid; i < nM; i += nthr) sM[i] = Mp[i];
  for (int i = tid; i < N; i += nthr) sw[i] = w[i];
  Linv = sL;
  Cin = sC;
  Mp = sM;
  w = sw;
}

// Zero the grid barrier's arrival count (grid_barrier_count) before a cooperative
// multi-sweep launch; one thread.
static __global__ void k_zero_gcount(unsigned long long *c) { *c = 0ull; }

// Fixed-order block sum of per-thread values (the result in thread 0).
__device__ __forceinline__ double block_reduce_fixed(float e2, double *red, int tid, int nthr) {
  double v = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read by a previous reduction
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  return bs;
}

// ---- cell-column loads and the structured FP32 cell solve of the two-sweep kernels
// Global loads of one cell column of a tile (z, the old correction when
// want_old, the lagged inflows from delta_in); zeros for an inactive thread.
template <int T, int NP, int PS, int GS>
__device__ __forceinline__ void ms2_load(float (&zr)[NP][4], float (&old)[NP][4], float (&uk)[NP], float (&uh)[NP],
                                         int tile, int cl, bool active, bool want_old, int J, int Nr, int Gr, int gy,
                                         bool zero, const float *__restrict__ z, const float *__restrict__ Din) {
  const int N = PS ? PS * NP : Nr, G = GS ? GS : Gr;
  const int P = N / NP, R = 4 * N * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int N2 = N / 2;
  const int offL = cl > 0 ? -1 : (T - 1) - R * T;
  const int offR = cl < T - 1 ? 1 : R * T - (T - 1);
  const int j = tile * T + cl;
  const size_t off = ((size_t)tile * R + (size_t)(g * N + m0) * 4) * T + cl;
  const float *__restrict__ zb = z + off;
  const float *__restrict__ db = Din + off;
#pragma unroll
  for (int i = 0; i < NP; i++) {
    const int m = m0 + i;
#pragma unroll
    for (int p = 0; p < 4; p++) {
      zr[i][p] = active ? zb[(i * 4 + p) * T] : 0.f;
      old[i][p] = (active && want_old && !zero) ? db[(i * 4 + p) * T] : 0.f;
    }
    uk[i] = 0.f;
    uh[i] = 0.f;
    if (active && !zero) {
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
}

// Structured FP32 cell solve of the thread's (cell, group, NP angles):
// t = z + Cin u, y = sum_m w t, s = Mp y, o = t + Linv s (the arithmetic of
// tiled_compute).  Three block barriers; y_s / yr_s / s_s as there.
template <int T, int NP, int PS, int GS>
__device__ __forceinline__ void ms2_solve(float (&o)[NP][4], const float (&zr)[NP][4], const float (&uk)[NP],
                                          const float (&uh)[NP], bool active, int tau, int Nr, int Gr, int cl, int gy,
                                          const float *Linv, const float *Cin, const float *Mp, const float *w,
                                          float *y_s, float *yr_s, float *s_s) {
  const int N = PS ? PS * NP : Nr, G = GS ? GS : Gr;
  const int P = N / NP, G4 = 4 * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int tb = tau * G * N;
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
#pragma unroll
  for (int i = 0; i < NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) o[i][p] = 0.f;
  if (active) {
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const float4 *C4 = reinterpret_cast<const float4 *>(Cin + (tb + g * N + m) * 8);
      const float4 ca = C4[0], cb = C4[1];
      o[i][0] = fmaf(ca.y, uh[i], fmaf(ca.x, uk[i], zr[i][0]));
      o[i][1] = fmaf(ca.w, uh[i], fmaf(ca.z, uk[i], zr[i][1]));
      o[i][2] = fmaf(cb.y, uh[i], fmaf(cb.x, uk[i], zr[i][2]));
      o[i][3] = fmaf(cb.w, uh[i], fmaf(cb.z, uk[i], zr[i][3]));
      const float wm = w[m];
      y0 = fmaf(wm, o[i][0], y0);
      y1 = fmaf(wm, o[i][1], y1);
      y2 = fmaf(wm, o[i][2], y2);
      y3 = fmaf(wm, o[i][3], y3);
    }
  }
  {
    float *ys = y_s + (gy * 4) * T + cl;
    ys[0] = y0;
    ys[T] = y1;
    ys[2 * T] = y2;
    ys[3 * T] = y3;
  }
  __syncthreads();
#pragma unroll
  for (int q = ch; q < 4; q += P) {
    float v = y_s[((g * P) * 4 + q) * T + cl];
#pragma unroll
    for (int k = 1; k < P; k++) v += y_s[((g * P + k) * 4 + q) * T + cl];
    yr_s[(g * 4 + q) * T + cl] = v;
  }
  __syncthreads();
  if (active)
#pragma unroll
    for (int q = ch; q < 4; q += P) {
      const float *M = Mp + tau * G4 * G4 + (g * 4 + q) * G4;
      float v = 0.f;
#pragma unroll
      for (int k = 0; k < G4; k++) v = fmaf(M[k], yr_s[k * T + cl], v);
      s_s[(g * 4 + q) * T + cl] = v;
    }
  __syncthreads();
  if (active) {
    const float s0 = s_s[(g * 4 + 0) * T + cl], s1 = s_s[(g * 4 + 1) * T + cl];
    const float s2 = s_s[(g * 4 + 2) * T + cl], s3 = s_s[(g * 4 + 3) * T + cl];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const float4 *L4 = reinterpret_cast<const float4 *>(Linv + (tb + g * N + m0 + i) * 16);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float4 L = L4[p];
        o[i][p] = fmaf(L.w, s3, fmaf(L.z, s2, fmaf(L.y, s1, fmaf(L.x, s0, o[i][p]))));
      }
    }
  }
}

// The downstream edge values of a cell (mu > 0: corners 1, 3; mu < 0: corners
// 0, 2) at edge[((g N + m) 2 + q)] (the run's outside neighbours).
template <int NP>
__device__ __forceinline__ void ms2_put_edges(float *edge, const float (&o)[NP][4], int N, int g, int m0) {
#pragma unroll
  for (int i = 0; i < NP; i++) {
    const int m = m0 + i;
    float *d = edge + (g * N + m) * 2;
    if (m >= N / 2) {
      d[0] = o[i][1];
      d[1] = o[i][3];
    } else {
      d[0] = o[i][0];
      d[1] = o[i][2];
    }
  }
}

// sum of squared changes
template <int NP>
__device__ __forceinline__ float ms2_dist2(const float (&a)[NP][4], const float (&b)[NP][4]) {
  float e2 = 0.f;
#pragma unroll
  for (int i = 0; i < NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) {
      const float d = a[i][p] - b[i][p];
      e2 = fmaf(d, d, e2);
    }
  return e2;
}

}  // namespace oci
