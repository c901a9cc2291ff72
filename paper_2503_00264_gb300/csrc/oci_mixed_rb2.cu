// oci_mixed_rb2.cu -- FP32 inner sweeps of the mixed form in red-black order,
// two sweeps per pass over the correction.
#include <math.h>

#include <algorithm>

#include "oci_device.cuh"
#include "oci_mixed_dev.cuh"

namespace oci {

// ---------------------------------------------------------------- inner sweeps, red-black, two per pass
// Two red-black sweeps (i, i+1) in one pass over the correction, by the run
// walk of the Jacobi form: at step k a block computes red^i on tile k+1 (from
// delta^{i-1} in global memory), black^i on tile k, red^{i+1} on tile k and
// black^{i+1} on tile k-1; every input is global delta^{i-1}, a half-tile of
// this pass kept in shared memory (red^i, black^i: two slots each, by tile
// parity), or red^{i+1} that the block itself has just written to the output.
// The cells next to the run whose values the walk needs are recomputed by the
// block: red^i and black^i of the two cells before it, red^i of the first two
// red cells after it, black^i between those and red^{i+1} of the first cell
// after it.  Results go to the other buffer (not in
// place: a neighbouring block still reads delta^{i-1} there), so one pass reads
// z and delta^{i-1} once and writes delta^{i+1} once; the device state takes
// the two norms in order, and when the first ends an inner block the sweep is
// recomputed by a one-sweep pass from the untouched input.  Same cell
// arithmetic and colour order as k_mx_rb; the correction arrays keep the
// colour-ordered tile-major layout.

// Lagged inflows of the thread's NP angles from the left neighbour (corners 1,
// 3; mu > 0) and the right neighbour (corners 0, 2; mu < 0).  L / Rt point at
// the neighbour's value in row (g N + m0) 4 of a column source with row stride
// ls / rs; nullptr is zero inflow.
template <int NP>
__device__ __forceinline__ void rb2_inflow(float (&uk)[NP], float (&uh)[NP], const float *L, int ls, const float *Rt,
                                           int rs, int m0, int N2) {
#pragma unroll
  for (int i = 0; i < NP; i++) {
    const int m = m0 + i;
    if (m >= N2) {
      uk[i] = L ? L[(i * 4 + 1) * ls] : 0.f;
      uh[i] = L ? L[(i * 4 + 3) * ls] : 0.f;
    } else {
      uk[i] = Rt ? Rt[(i * 4 + 0) * rs] : 0.f;
      uh[i] = Rt ? Rt[(i * 4 + 2) * rs] : 0.f;
    }
  }
}

template <int NP>
__device__ __forceinline__ void rb2_get(float (&v)[NP][4], const float *src, int st, bool act) {
#pragma unroll
  for (int i = 0; i < NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) v[i][p] = (act && src) ? src[(i * 4 + p) * st] : 0.f;
}

template <int NP>
__device__ __forceinline__ void rb2_put(float *dst, int st, const float (&v)[NP][4]) {
#pragma unroll
  for (int i = 0; i < NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) dst[(i * 4 + p) * st] = v[i][p];
}

struct Rb2Args {
  int J, N, G, t0, t1;
  const int32_t *__restrict__ type;
  const float *Linv, *Cin, *Mp, *w;
  const float *__restrict__ z;
  float *y_s, *yr_s, *s_s;
  float *Ri, *Bi;                              // two half-tile slots each ([R][T/2])
  float *hRL, *hBL, *hRR0, *hRR1, *hBR, *hR2;  // cells next to the run, [R] each
};

// One red-black pass over the block's run: ns = 2 sweeps i, i+1 (delta^{i+1}
// into Dout), or ns = 1 sweep i (delta^i into Dout).  ea, eb: the thread's
// squared changes of the two sweeps.
template <int T, int NP, int PS, int GS>
__device__ void rb2_pass(const Rb2Args &a, int cl, int gy, bool zero, int ns, const float *__restrict__ Din,
                         float *__restrict__ Dout, float &ea, float &eb) {
  constexpr int TH = T / 2;
  const int N = PS ? PS * NP : a.N, G = GS ? GS : a.G;
  const int J = a.J, P = N / NP, R = 4 * N * G, N2 = N / 2;
  const int g = gy / P, m0 = (gy % P) * NP, row0 = (g * N + m0) * 4;
  const int ntiles = (J + T - 1) / T, t0 = a.t0, t1 = a.t1;
  const size_t RT = (size_t)R * T;
  const int HS = R * TH;  // one half-tile slot
  // column c of colour col of a global tile, at row row0 (row stride T)
  auto gcol = [&](const float *base, int tile, int col, int c) -> const float * {
    return base + (size_t)tile * RT + (size_t)row0 * T + col * TH + c;
  };
  auto gout = [&](int tile, int col, int c) -> float * {
    return Dout + (size_t)tile * RT + (size_t)row0 * T + col * TH + c;
  };
  // column c of the slot of `tile` (by parity), at row row0 (row stride T/2)
  auto scol = [&](float *slot, int tile, int c) -> float * { return slot + (tile & 1) * HS + row0 * TH + c; };
  auto solve = [&](float (&o)[NP][4], const float (&zr)[NP][4], const float (&uk)[NP], const float (&uh)[NP],
                   bool act, int j) {
    const int tau = act ? a.type[j] : 0;
    ms2_solve<TH, NP, PS, GS>(o, zr, uk, uh, act, tau, N, G, cl, gy, a.Linv, a.Cin, a.Mp, a.w, a.y_s, a.yr_s,
                              a.s_s);
  };
  // inputs of red^i at (tile, c) from delta^{i-1}: inflows, z, old value
  auto red_i_in = [&](int tile, int c, bool act, float (&zr)[NP][4], float (&old)[NP][4], float (&uk)[NP],
                      float (&uh)[NP]) {
    const int j = tile * T + 2 * c;
    const float *L = nullptr, *Rt = nullptr;
    if (act && !zero) {
      if (c > 0) L = gcol(Din, tile, 1, c - 1);
      else if (j > 0) L = gcol(Din, tile - 1, 1, TH - 1);
      if (j + 1 < J) Rt = gcol(Din, tile, 1, c);
    }
    rb2_inflow<NP>(uk, uh, L, T, Rt, T, m0, N2);
    rb2_get<NP>(zr, gcol(a.z, tile, 0, c), T, act);
    rb2_get<NP>(old, zero ? nullptr : gcol(Din, tile, 0, c), T, act);
  };
  // --- reds of sweep i next to the run: column T/2-1 takes red (t0-1, T/2-1),
  // columns 0 and 1 take reds (t1, 0) and (t1, 1)
  {
    int tile = t0;
    bool act = false;
    float *dst = nullptr;
    if (cl == TH - 1 && t0 > 0 && ns == 2) {
      tile = t0 - 1;
      act = true;
      dst = a.hRL;
    } else if (cl == 0 && t1 < ntiles) {
      tile = t1;
      act = true;
      dst = a.hRR0;
    } else if (cl == 1 && ns == 2 && t1 < ntiles && t1 * T + 2 < J) {
      tile = t1;
      act = true;
      dst = a.hRR1;
    }
    float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
    red_i_in(tile, cl, act, zr, old, uk, uh);
    solve(o, zr, uk, uh, act, tile * T + 2 * cl);
    if (act) rb2_put<NP>(dst + row0, 1, o);
  }
  // --- red^i of tile t0
  {
    const int j = t0 * T + 2 * cl;
    const bool act = j < J;
    float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
    red_i_in(t0, cl, act, zr, old, uk, uh);
    solve(o, zr, uk, uh, act, j);
    if (act) {
      ea += ms2_dist2<NP>(o, old);
      rb2_put<NP>(scol(a.Ri, t0, cl), TH, o);
      if (ns == 1) rb2_put<NP>(gout(t0, 0, cl), T, o);
    }
  }
  __syncthreads();
  // --- blacks of sweep i next to the run: black (t0-1, T/2-1) and black (t1, 0)
  if (ns == 2) {
    const bool bl = cl == TH - 1 && t0 > 0;
    const int jr = t1 * T + 1;
    const bool br = cl == 0 && t1 < ntiles && jr < J;
    const bool act = bl || br;
    const float *L = nullptr, *Rt = nullptr;
    int tile = t0, col = 0, j = 0, rs = 1;
    if (bl) {
      tile = t0 - 1;
      col = TH - 1;
      j = t0 * T - 1;
      L = a.hRL + row0;
      Rt = scol(a.Ri, t0, 0);
      rs = TH;
    } else if (br) {
      tile = t1;
      col = 0;
      j = jr;
      L = a.hRR0 + row0;
      Rt = jr + 1 < J ? a.hRR1 + row0 : nullptr;
    }
    float zr[NP][4], uk[NP], uh[NP], o[NP][4];
    rb2_inflow<NP>(uk, uh, L, 1, Rt, rs, m0, N2);
    rb2_get<NP>(zr, gcol(a.z, tile, 1, col), T, act);
    solve(o, zr, uk, uh, act, j);
    if (bl) rb2_put<NP>(a.hBL + row0, 1, o);
    if (br) rb2_put<NP>(a.hBR + row0, 1, o);
  }
  for (int k = t0; k < t1; k++) {
    if (k + 1 < t1) {  // (a) red^i of tile k+1
      const int j = (k + 1) * T + 2 * cl;
      const bool act = j < J;
      float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
      red_i_in(k + 1, cl, act, zr, old, uk, uh);
      solve(o, zr, uk, uh, act, j);
      if (act) {
        ea += ms2_dist2<NP>(o, old);
        rb2_put<NP>(scol(a.Ri, k + 1, cl), TH, o);
        if (ns == 1) rb2_put<NP>(gout(k + 1, 0, cl), T, o);
      }
    }
    __syncthreads();
    {  // (b) black^i of tile k
      const int j = k * T + 2 * cl + 1;
      const bool act = j < J;
      const float *L = nullptr, *Rt = nullptr;
      int rs = TH;
      if (act) {
        L = scol(a.Ri, k, cl);
        if (j + 1 < J) {
          if (cl + 1 < TH) Rt = scol(a.Ri, k, cl + 1);
          else if (k + 1 < t1) Rt = scol(a.Ri, k + 1, 0);
          else Rt = a.hRR0 + row0, rs = 1;
        }
      }
      float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
      rb2_inflow<NP>(uk, uh, L, TH, Rt, rs, m0, N2);
      rb2_get<NP>(zr, gcol(a.z, k, 1, cl), T, act);
      rb2_get<NP>(old, zero ? nullptr : gcol(Din, k, 1, cl), T, act);
      solve(o, zr, uk, uh, act, j);
      if (act) {
        ea += ms2_dist2<NP>(o, old);
        if (ns == 2) rb2_put<NP>(scol(a.Bi, k, cl), TH, o);
        else rb2_put<NP>(gout(k, 1, cl), T, o);
      }
    }
    if (ns == 1) continue;
    __syncthreads();
    {  // (c) red^{i+1} of tile k
      const int j = k * T + 2 * cl;
      const bool act = j < J;
      const float *L = nullptr, *Rt = nullptr;
      int ls = TH;
      if (act) {
        if (cl > 0) L = scol(a.Bi, k, cl - 1);
        else if (j > 0) {
          if (k > t0) L = scol(a.Bi, k - 1, TH - 1);
          else L = a.hBL + row0, ls = 1;
        }
        if (j + 1 < J) Rt = scol(a.Bi, k, cl);
      }
      float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
      rb2_inflow<NP>(uk, uh, L, ls, Rt, TH, m0, N2);
      rb2_get<NP>(zr, gcol(a.z, k, 0, cl), T, act);
      rb2_get<NP>(old, scol(a.Ri, k, cl), TH, act);
      solve(o, zr, uk, uh, act, j);
      if (act) {
        eb += ms2_dist2<NP>(o, old);
        rb2_put<NP>(gout(k, 0, cl), T, o);
      }
    }
    if (k > t0) {  // (d) black^{i+1} of tile k-1
      __syncthreads();
      const int kk = k - 1, j = kk * T + 2 * cl + 1;
      const bool act = j < J;
      const float *L = nullptr, *Rt = nullptr;
      if (act) {  // red^{i+1} of tiles k-1 and k: written to Dout by this block at (c)
        L = gcol(Dout, kk, 0, cl);
        if (j + 1 < J) Rt = cl + 1 < TH ? gcol(Dout, kk, 0, cl + 1) : gcol(Dout, k, 0, 0);
      }
      float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
      rb2_inflow<NP>(uk, uh, L, T, Rt, T, m0, N2);
      rb2_get<NP>(zr, gcol(a.z, kk, 1, cl), T, act);
      rb2_get<NP>(old, scol(a.Bi, kk, cl), TH, act);
      solve(o, zr, uk, uh, act, j);
      if (act) {
        eb += ms2_dist2<NP>(o, old);
        rb2_put<NP>(gout(kk, 1, cl), T, o);
      }
    }
  }
  if (ns == 1) return;
  __syncthreads();
  {  // red^{i+1} of cell t1*T (column 0 of tile t1), for the run's last black cell
    const int j = t1 * T;
    const bool act = cl == 0 && t1 < ntiles;
    const float *L = nullptr, *Rt = nullptr;
    if (act) {
      L = scol(a.Bi, t1 - 1, TH - 1);
      if (j + 1 < J) Rt = a.hBR + row0;
    }
    float zr[NP][4], uk[NP], uh[NP], o[NP][4];
    rb2_inflow<NP>(uk, uh, L, TH, Rt, 1, m0, N2);
    rb2_get<NP>(zr, gcol(a.z, act ? t1 : t0, 0, 0), T, act);
    solve(o, zr, uk, uh, act, j);
    if (act) rb2_put<NP>(a.hR2 + row0, 1, o);
  }
  __syncthreads();
  {  // black^{i+1} of tile t1-1
    const int kk = t1 - 1, j = kk * T + 2 * cl + 1;
    const bool act = j < J;
    const float *L = nullptr, *Rt = nullptr;
    int rs = T;
    if (act) {
      L = gcol(Dout, kk, 0, cl);
      if (j + 1 < J) {
        if (cl + 1 < TH) Rt = gcol(Dout, kk, 0, cl + 1);
        else Rt = a.hR2 + row0, rs = 1;
      }
    }
    float zr[NP][4], old[NP][4], uk[NP], uh[NP], o[NP][4];
    rb2_inflow<NP>(uk, uh, L, T, Rt, rs, m0, N2);
    rb2_get<NP>(zr, gcol(a.z, kk, 1, cl), T, act);
    rb2_get<NP>(old, scol(a.Bi, kk, cl), TH, act);
    solve(o, zr, uk, uh, act, j);
    if (act) {
      eb += ms2_dist2<NP>(o, old);
      rb2_put<NP>(gout(kk, 1, cl), T, o);
    }
  }
}

// block size (when fixed at compile time) and resident blocks the registers are built for
template <int T, int PS, int GS>
struct Rb2Bounds {
  static constexpr int thr = (PS && GS) ? T / 2 * PS * GS : 256;
  static constexpr int minb = 512 / thr > 0 ? 512 / thr : 1;
};

template <int T, int NP, int PS, int GS>
__global__ void __launch_bounds__(Rb2Bounds<T, PS, GS>::thr, Rb2Bounds<T, PS, GS>::minb)
    k_mx_rb2(int J, int N, int G, int n_types, int stage, const int32_t *__restrict__ type, const float *Linv_g,
             const float *Cin_g, const float *Mp_g, const float *w_g, const float *__restrict__ z, float *D0,
             float *D1, DevState *ds, double *__restrict__ partials, unsigned long long *gbar, double *e_hist,
             cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  constexpr int TH = T / 2;
  extern __shared__ __align__(16) float smr[];
  __shared__ double red[8];
  __shared__ DevState sd;
  __shared__ int s_ok, s_roll;
  unsigned long long gep = 0;  // thread 0: the arrival count the next grid barrier waits for
  const int P = N / NP, G4 = 4 * G, R = 4 * N * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the grid
  Rb2Args a;
  a.J = J;
  a.N = N;
  a.G = G;
  a.type = type;
  a.z = z;
  a.y_s = smr;
  a.yr_s = a.y_s + (size_t)G * P * 4 * TH;
  a.s_s = a.yr_s + (size_t)G4 * TH;
  a.Ri = a.s_s + (size_t)G4 * TH;
  a.Bi = a.Ri + (size_t)2 * R * TH;
  a.hRL = a.Bi + (size_t)2 * R * TH;
  a.hBL = a.hRL + R;
  a.hRR0 = a.hBL + R;
  a.hRR1 = a.hRR0 + R;
  a.hBR = a.hRR1 + R;
  a.hR2 = a.hBR + R;
  a.Linv = Linv_g;
  a.Cin = Cin_g;
  a.Mp = Mp_g;
  a.w = w_g;
  if (stage) {
    stage_tables(a.hR2 + R, n_types, N, G, tid, nthr, a.Linv, a.Cin, a.Mp, a.w);
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
    rb2_pass<T, NP, PS, GS>(a, cl, gy, zero, ns, Din, Dout, ea, eb);
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
          s_roll = 1;  // the inner block ends at sweep i
        } else {
          finish_mixed(&sd, eh, sqrt(tb), cond, 0);
          if (!sd.inplace) sd.dcur ^= 1;  // one buffer flip per pass
        }
      }
    }
    __syncthreads();
    if (s_roll) {  // sweep i alone into Dout (delta^{i-1} is untouched in Din)
      float x = 0.f, y = 0.f;
      rb2_pass<T, NP, PS, GS>(a, cl, gy, zero, 1, Din, Dout, x, y);
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

size_t mx_rb2_smem(const Handle &h, int T, int P, bool stage) {
  const size_t G = h.G, N = h.N, TH = T / 2, R = 4 * N * G;
  return ((size_t)TH * (G * P * 4 + 8 * G) + 4 * R * TH + 6 * R) * 4 + (stage ? mx_tables_floats(h) * 4 + 16 : 0);
}

template <int T, int NP, int PS, int GS>
static void launch_rb2(Handle &h, int P, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
  const size_t smem = mx_rb2_smem(h, T, P, stage);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_rb2<T, NP, PS, GS>, (T / 2) * h.G * P, smem);
  const int ntiles = (h.J + T - 1) / T;
  const int grid = std::min(sms * per, ntiles);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T / 2, h.G * P);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  k_zero_gcount<<<1, 1, 0, h.stream>>>(reinterpret_cast<unsigned long long *>(h.gbar));
  cudaLaunchKernelEx(&cfg, k_mx_rb2<T, NP, PS, GS>, h.J, h.N, h.G, h.tt.n_types, (int)stage,
                     (const int32_t *)h.type, (const float *)h.tt.Linv32, (const float *)h.tt.Cin32,
                     (const float *)h.tt.Mp32, (const float *)h.w32, (const float *)h.z32, h.delta[0], h.delta[1],
                     h.ds, h.partials, reinterpret_cast<unsigned long long *>(h.gbar), h.e_hist, cond, use_cond, max_sweeps);
}

// S16, one group: angle chunks and groups fixed at compile time; else generic
void launch_rb2_any(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const int T = h.mx_cb, P = h.mx_P, np = h.N / P;
  const bool s16 = h.N == 16 && h.G == 1;
#define OCI_RB2(TT, NPP)                                                         \
  do {                                                                           \
    if (s16) launch_rb2<TT, NPP, 16 / NPP, 1>(h, P, cond, use_cond, max_sweeps); \
    else launch_rb2<TT, NPP, 0, 0>(h, P, cond, use_cond, max_sweeps);            \
  } while (0)
  if (T == 32) {
    if (np == 2) OCI_RB2(32, 2);
    else OCI_RB2(32, 4);
  } else {
    if (np == 2) OCI_RB2(64, 2);
    else OCI_RB2(64, 4);
  }
#undef OCI_RB2
}

// Dynamic shared memory limits of the kernels above 48 KB (set once at setup).
int mx_rb2_set_attributes() {
  const void *ks[] = {(const void *)k_mx_rb2<32, 2, 0, 0>, (const void *)k_mx_rb2<32, 4, 0, 0>,
                      (const void *)k_mx_rb2<64, 2, 0, 0>, (const void *)k_mx_rb2<64, 4, 0, 0>,
                      (const void *)k_mx_rb2<32, 2, 8, 1>, (const void *)k_mx_rb2<32, 4, 4, 1>,
                      (const void *)k_mx_rb2<64, 2, 8, 1>, (const void *)k_mx_rb2<64, 4, 4, 1>};
  for (const void *k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(red-black two-sweep FP32 inner sweep)");
  }
  return OCI_OK;
}

}  // namespace oci
