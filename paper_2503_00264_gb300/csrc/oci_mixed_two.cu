// oci_mixed_two.cu -- FP32 inner sweeps of the mixed form that advance the
// correction by two Jacobi sweeps per pass over it.
#include <math.h>

#include <algorithm>

#include "oci_device.cuh"
#include "oci_mixed_dev.cuh"

namespace oci {

// ---------------------------------------------------------------- inner sweeps, two per pass
// Two consecutive inner sweeps in one pass over the correction (temporal
// blocking).  Each block owns a contiguous run of tiles [t0, t1) and walks it
// left to right: at step k it computes delta^{i+1} on tile k from delta^i in
// global memory, then delta^{i+2} on tile k-1, whose lagged inflows are the
// delta^{i+1} values of tiles k-2, k-1 and k held in a three-slot ring in
// shared memory.  The delta^{i+1} values of the two cells just outside the run
// (t0 T - 1 and t1 T) are recomputed by the block before the walk, so blocks never
// wait on one another inside a pass.  Per two sweeps a pass reads z and
// delta^i once and writes delta^{i+2} once: 12 bytes per unknown instead of
// 24.  Both sweeps' norms are reduced and the device state takes the two e
// values in order; if the first already ends the inner block (a refinement or
// the stop rule is due), delta^{i+1} is recomputed from delta^i -- still intact
// in the input buffer -- by a one-sweep pass into the output buffer.  The cell
// arithmetic is that of the tiled sweep.
//
// Template parameters: T cells per tile, NP angles per thread, and the angle
// chunks per cell PS and groups GS when known at compile time (0: taken from
// the arguments); with both fixed every index and loop bound folds.

struct Ms2Args {
  int J, N, G, t0, t1;
  const int32_t *__restrict__ type;
  const float *Linv, *Cin, *Mp, *w;
  const float *__restrict__ z;
  float *y_s, *yr_s, *s_s, *ring, *halo;
};

// The next tile's z and correction (two contiguous chunks of 4NG*T floats in the
// tile-major layout) into L1 while this tile is solved: one prefetch per thread
// and 128-byte line, no registers held.
template <int T>
__device__ __forceinline__ void ms2_prefetch_tile(const float *z, const float *Din, int tile, int R, int tid,
                                                  int nthr) {
  const int lines = R * T / 32;
  const size_t base = (size_t)tile * R * T;
  for (int l = tid; l < 2 * lines; l += nthr) {
    const float *p = (l < lines ? z : Din) + base + (size_t)(l < lines ? l : l - lines) * 32;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
  }
}

// One sweep over the block's run (delta_in -> delta_out); returns the thread's
// sum of squared changes.
template <int T, int NP, int PS, int GS>
__device__ float ms2_pass1(const Ms2Args &a, int cl, int gy, bool zero, const float *__restrict__ Din,
                           float *__restrict__ Dout) {
  const int N = PS ? PS * NP : a.N, G = GS ? GS : a.G;
  const int P = N / NP, R = 4 * N * G;
  const int g = gy / P, m0 = (gy % P) * NP;
  float e2 = 0.f;
  for (int k = a.t0; k < a.t1; k++) {
    if (k + 1 < a.t1) ms2_prefetch_tile<T>(a.z, Din, k + 1, R, gy * T + cl, T * P * G);
    float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
    const int j = k * T + cl;
    const bool act = j < a.J;
    const int tau = act ? a.type[j] : 0;
    ms2_load<T, NP, PS, GS>(zr, old, uk, uh, k, cl, act, true, a.J, N, G, gy, zero, a.z, Din);
    ms2_solve<T, NP, PS, GS>(o, zr, uk, uh, act, tau, N, G, cl, gy, a.Linv, a.Cin, a.Mp, a.w, a.y_s, a.yr_s,
                             a.s_s);
    if (act) {
      e2 += ms2_dist2<NP>(o, old);
      float *__restrict__ ob = Dout + ((size_t)k * R + (size_t)(g * N + m0) * 4) * T + cl;
#pragma unroll
      for (int i = 0; i < NP; i++)
#pragma unroll
        for (int p = 0; p < 4; p++) ob[(i * 4 + p) * T] = o[i][p];
    }
  }
  return e2;
}

// Two sweeps over the block's run (delta_in -> delta_out = delta^{i+2}); the
// threads' sums of squared changes of both sweeps in ea, eb.  delta^{i+1} of a
// tile is kept whole in a ring slot [4NG][T] (for the second sweep's norm and
// its inflows); z is read again for the second sweep (a cache hit: the tile
// was read one step earlier).
template <int T, int NP, int PS, int GS>
__device__ void ms2_pass2(const Ms2Args &a, int cl, int gy, bool zero, const float *__restrict__ Din,
                          float *__restrict__ Dout, float &ea, float &eb) {
  const int N = PS ? PS * NP : a.N, G = GS ? GS : a.G;
  const int J = a.J, P = N / NP, R = 4 * N * G, NG2 = 2 * N * G;
  const int g = gy / P, m0 = (gy % P) * NP;
  const int ntiles = (J + T - 1) / T;
  float *halo_l = a.halo, *halo_r = a.halo + NG2;
  // delta^{i+1} of the cells next to the run: thread column T-1 takes cell
  // t0*T - 1 (last column of tile t0-1), column 0 takes cell t1*T (tile t1)
  {
    const bool hl = cl == T - 1 && a.t0 > 0, hr = cl == 0 && a.t1 < ntiles;
    const bool act = hl || hr;
    const int tile = hl ? a.t0 - 1 : (hr ? a.t1 : a.t0);
    const int tau = act ? a.type[tile * T + cl] : 0;
    float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
    ms2_load<T, NP, PS, GS>(zr, old, uk, uh, tile, cl, act, false, J, N, G, gy, zero, a.z, Din);
    ms2_solve<T, NP, PS, GS>(o, zr, uk, uh, act, tau, N, G, cl, gy, a.Linv, a.Cin, a.Mp, a.w, a.y_s, a.yr_s,
                             a.s_s);
    if (hl) ms2_put_edges<NP>(halo_l, o, N, g, m0);
    if (hr) ms2_put_edges<NP>(halo_r, o, N, g, m0);
  }
  // ring slots of tiles k (cur), k-1 (prv) and k-2 (pp)
  float *cur = a.ring, *prv = a.ring + R * T, *pp = a.ring + 2 * R * T;
  for (int k = a.t0; k <= a.t1; k++) {
    if (k + 1 < a.t1) ms2_prefetch_tile<T>(a.z, Din, k + 1, R, gy * T + cl, T * P * G);
    if (k < a.t1) {  // sweep i+1 on tile k
      float zr[NP][4], old[NP][4], uk[NP], uh[NP], o1[NP][4];
      const int j = k * T + cl;
      const bool act = j < J;
      const int tau = act ? a.type[j] : 0;
      ms2_load<T, NP, PS, GS>(zr, old, uk, uh, k, cl, act, true, J, N, G, gy, zero, a.z, Din);
      ms2_solve<T, NP, PS, GS>(o1, zr, uk, uh, act, tau, N, G, cl, gy, a.Linv, a.Cin, a.Mp, a.w, a.y_s, a.yr_s,
                               a.s_s);
      if (act) {
        ea += ms2_dist2<NP>(o1, old);
        float *sl = cur + ((g * N + m0) * 4) * T + cl;
#pragma unroll
        for (int i = 0; i < NP; i++)
#pragma unroll
          for (int p = 0; p < 4; p++) sl[(i * 4 + p) * T] = o1[i][p];
      }
    }
    __syncthreads();  // the ring slot of tile k is complete
    if (k > a.t0) {   // sweep i+2 on tile k-1: inflows from delta^{i+1} of the neighbours
      const int kk = k - 1, j = kk * T + cl;
      const bool act = j < J;
      const int tau = act ? a.type[j] : 0;
      float zr[NP][4], o1[NP][4], uk[NP], uh[NP], o2[NP][4];
      {
        float dummy[NP][4], dk[NP], dh[NP];
        ms2_load<T, NP, PS, GS>(zr, dummy, dk, dh, kk, cl, act, false, J, N, G, gy, true, a.z, Din);
      }
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const int m = m0 + i, r0 = (g * N + m) * 4;
#pragma unroll
        for (int p = 0; p < 4; p++) o1[i][p] = act ? prv[(r0 + p) * T + cl] : 0.f;
        const float *src = nullptr;
        int st = 2 * T;
        if (m >= N / 2) {  // corners 1, 3 of cell j - 1
          if (j > 0) {
            if (cl > 0) src = prv + (r0 + 1) * T + cl - 1;
            else if (kk > a.t0) src = pp + (r0 + 1) * T + T - 1;
            else src = halo_l + (g * N + m) * 2, st = 1;
          }
        } else if (j < J - 1) {  // corners 0, 2 of cell j + 1
          if (cl < T - 1) src = prv + r0 * T + cl + 1;
          else if (kk + 1 < a.t1) src = cur + r0 * T;
          else src = halo_r + (g * N + m) * 2, st = 1;
        }
        uk[i] = (act && src) ? src[0] : 0.f;
        uh[i] = (act && src) ? src[st] : 0.f;
      }
      ms2_solve<T, NP, PS, GS>(o2, zr, uk, uh, act, tau, N, G, cl, gy, a.Linv, a.Cin, a.Mp, a.w, a.y_s, a.yr_s,
                               a.s_s);
      if (act) {
        eb += ms2_dist2<NP>(o2, o1);
        float *__restrict__ ob = Dout + ((size_t)kk * R + (size_t)(g * N + m0) * 4) * T + cl;
#pragma unroll
        for (int i = 0; i < NP; i++)
#pragma unroll
          for (int p = 0; p < 4; p++) ob[(i * 4 + p) * T] = o2[i][p];
      }
    }
    float *t = pp;  // rotate: the slot of tile k-2 takes tile k+1
    pp = prv;
    prv = cur;
    cur = t;
  }
}

// OCC: resident blocks per SM the register allocation is built for (the
// block size is T * PS * GS threads when known at compile time, else <= 256).
template <int T, int NP, int PS, int GS, int OCC>
__global__ void __launch_bounds__((PS && GS) ? T * PS * GS : 256, OCC)
    k_mx_inner_ms2(int J, int N, int G, int n_types, int stage, const int32_t *__restrict__ type, const float *Linv_g,
                   const float *Cin_g, const float *Mp_g, const float *w_g, const float *__restrict__ z, float *D0,
                   float *D1, DevState *ds, double *__restrict__ partials, unsigned long long *gbar, double *e_hist,
                   cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  extern __shared__ __align__(16) float smr[];
  __shared__ double red[8];
  __shared__ DevState sd;
  __shared__ int s_ok, s_roll;
  unsigned long long gep = 0;  // thread 0: the arrival count the next grid barrier waits for
  const int P = N / NP, G4 = 4 * G, NG2 = 2 * N * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the grid
  Ms2Args a;
  a.J = J;
  a.N = N;
  a.G = G;
  a.type = type;
  a.z = z;
  a.y_s = smr;
  a.yr_s = a.y_s + (size_t)G * P * 4 * T;
  a.s_s = a.yr_s + (size_t)G4 * T;
  a.ring = a.s_s + (size_t)G4 * T;
  a.halo = a.ring + (size_t)3 * 4 * N * G * T;
  a.Linv = Linv_g;
  a.Cin = Cin_g;
  a.Mp = Mp_g;
  a.w = w_g;
  if (stage) {
    stage_tables(a.halo + 2 * NG2, n_types, N, G, tid, nthr, a.Linv, a.Cin, a.Mp, a.w);
    __syncthreads();
  }
  const int ntiles = (J + T - 1) / T;
  a.t0 = (int)((long long)blockIdx.x * ntiles / gridDim.x);
  a.t1 = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
  bool failed = false;
  for (int sw = 0, pass = 0;; pass++) {
    const int ns = max_sweeps - sw >= 2 ? 2 : 1;
    const bool zero = sd.refine || sd.blk_i == 0;
    const float *__restrict__ Din = sd.dcur ? D1 : D0;
    float *__restrict__ Dout = sd.dcur ? D0 : D1;
    float ea = 0.f, eb = 0.f;
    if (ns == 2) ms2_pass2<T, NP, PS, GS>(a, cl, gy, zero, Din, Dout, ea, eb);
    else ea = ms2_pass1<T, NP, PS, GS>(a, cl, gy, zero, Din, Dout);
    const double ba = block_reduce_fixed(ea, red, tid, nthr);
    const double bb = block_reduce_fixed(eb, red, tid, nthr);
    double *part = partials + (size_t)(pass & 1) * 2 * gridDim.x;
    if (tid == 0) {
      part[blockIdx.x] = ba;
      part[gridDim.x + blockIdx.x] = bb;
      s_ok = grid_barrier_count(gbar, gep += gridDim.x, sd.spin);
    }
    __syncthreads();
    if (!s_ok) {
      failed = true;
      break;
    }
    const double ta = block_sum_fixed(part, gridDim.x, red);
    const double tb = ns == 2 ? block_sum_fixed(part + gridDim.x, gridDim.x, red) : 0.0;
    if (tid == 0) {
      double *eh = blockIdx.x == 0 ? e_hist : nullptr;
      finish_mixed(&sd, eh, sqrt(ta), cond, 0);
      s_roll = 0;
      if (ns == 2) {
        if (sd.done || sd.refine) {
          s_roll = 1;  // the inner block ends at sweep i+1
        } else {
          finish_mixed(&sd, eh, sqrt(tb), cond, 0);
          if (!sd.inplace) sd.dcur ^= 1;  // one buffer flip per pass: delta^{i+2} is in Dout
        }
      }
    }
    __syncthreads();
    if (s_roll) {  // delta^{i+1} into Dout (delta^i is untouched in Din)
      ms2_pass1<T, NP, PS, GS>(a, cl, gy, zero, Din, Dout);
      break;
    }
    sw += ns;
    if (sd.done || sd.refine || sw >= max_sweeps) break;  // uniform: every block holds the same state
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

size_t mx_ms2_smem(const Handle &h, int T, int P, bool stage) {
  const size_t G = h.G, N = h.N;
  return ((size_t)T * (G * P * 4 + 8 * G) + 3 * 4 * N * G * T + 4 * N * G) * 4 +
         (stage ? mx_tables_floats(h) * 4 + 16 : 0);
}

template <int T, int NP, int PS, int GS, int OCC>
static void launch_ms2(Handle &h, int P, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
  const size_t smem = mx_ms2_smem(h, T, P, stage);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_ms2<T, NP, PS, GS, OCC>, T * h.G * P, smem);
  const int ntiles = (h.J + T - 1) / T;
  const int grid = std::min(sms * per, ntiles);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T, h.G * P);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  k_zero_gcount<<<1, 1, 0, h.stream>>>(reinterpret_cast<unsigned long long *>(h.gbar));
  cudaLaunchKernelEx(&cfg, k_mx_inner_ms2<T, NP, PS, GS, OCC>, h.J, h.N, h.G, h.tt.n_types, (int)stage,
                     (const int32_t *)h.type, (const float *)h.tt.Linv32, (const float *)h.tt.Cin32,
                     (const float *)h.tt.Mp32, (const float *)h.w32, (const float *)h.z32, h.delta[0], h.delta[1],
                     h.ds, h.partials, reinterpret_cast<unsigned long long *>(h.gbar), h.e_hist, cond, use_cond, max_sweeps);
}

// S16, one group (the slab workloads): fully specialised, with registers for
// 2 blocks of 256 / 4 of 128 threads per SM, or (kMxTiled2Occ) for 3 of 256 /
// 5 of 128; everything else generic (2 blocks of up to 256 threads)
void launch_ms2_any(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
  const bool s16 = h.N == 16 && h.G == 1, occ = h.mx_kind == kMxTiled2Occ;
#define OCI_MS2(TT, NPP, OC, OCX)                                                              \
  do {                                                                                         \
    if (s16 && occ) launch_ms2<TT, NPP, 16 / NPP, 1, OCX>(h, P, cond, use_cond, max_sweeps);   \
    else if (s16) launch_ms2<TT, NPP, 16 / NPP, 1, OC>(h, P, cond, use_cond, max_sweeps);      \
    else launch_ms2<TT, NPP, 0, 0, 2>(h, P, cond, use_cond, max_sweeps);                       \
  } while (0)
  if (T == 32) {
    if (np == 2) OCI_MS2(32, 2, 2, 3);
    else OCI_MS2(32, 4, 4, 5);
  } else {
    if (np == 2) OCI_MS2(64, 2, 1, 1);  // 512 threads: not an S16 shape (no candidate)
    else OCI_MS2(64, 4, 2, 3);
  }
#undef OCI_MS2
}


// Dynamic shared memory limits of the kernels above 48 KB (set once at setup).
int mx_two_set_attributes() {
  const void *ks[] = {(const void *)k_mx_inner_ms2<32, 2, 0, 0, 2>, (const void *)k_mx_inner_ms2<32, 4, 0, 0, 2>,
                      (const void *)k_mx_inner_ms2<64, 2, 0, 0, 2>, (const void *)k_mx_inner_ms2<64, 4, 0, 0, 2>,
                      (const void *)k_mx_inner_ms2<32, 2, 8, 1, 2>, (const void *)k_mx_inner_ms2<32, 4, 4, 1, 4>,
                      (const void *)k_mx_inner_ms2<64, 2, 8, 1, 1>, (const void *)k_mx_inner_ms2<64, 4, 4, 1, 2>,
                      (const void *)k_mx_inner_ms2<32, 2, 8, 1, 3>, (const void *)k_mx_inner_ms2<32, 4, 4, 1, 5>,
                      (const void *)k_mx_inner_ms2<64, 4, 4, 1, 3>};
  for (const void *k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(two-sweep FP32 inner sweep)");
  }
  const int e = mx_rb2_set_attributes();
  return e != OCI_OK ? e : mx_w2_set_attributes();
}

}  // namespace oci
