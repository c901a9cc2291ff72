// oci_mixed_warp.cu -- FP32 inner sweeps of the mixed form, two per pass, with
// every warp walking its own run of cells (one energy group, N = 8, 16, 32).
//
// The inner sweep is delta^{i+1} = A~^{-1}(r + B delta^i) per cell through the
// structured FP32 solve t = z + Cin u, y = sum_m w t, s = Mp y, delta = t + Linv s
// (Eqs. Aj, scatter, fullOCIlhs restated for the correction; z = Linv r comes
// from the FP64 refinement).  Layout: the tile-major FP32 correction arrays
// [J/32][4N][32] of the tiled kernels.
//
// Lanes: P = N/4 lanes per cell (four angles each), CW = 32/P cells per warp
// step; lane = ch * CW + c holds cell c of the step, angles 4 ch .. 4 ch + 3.
// The angular sum y is a butterfly over the P lanes of a cell (warp shuffles),
// so a cell solve needs no block barrier.  Each warp owns a contiguous run of
// steps (groups of CW cells) [k0, k1) and walks it left to right: at step k it
// computes delta^{i+1} of group k from delta^i in global memory, then
// delta^{i+2} of group k-1, whose lagged inflows are delta^{i+1} of its
// neighbours, read from a per-warp ring in shared memory that holds
// delta^{i+1} of groups k, k-1 and k-2:
//   - mu > 0 (corners 1, 3 of cell j-1): the lane one to the left, or for the
//     group's first cell the last cell of group k-2;
//   - mu < 0 (corners 0, 2 of cell j+1): the lane one to the right, or for the
//     group's last cell the first cell of group k.
// delta^{i+1} of the two cells just outside the run is recomputed by the warp
// before the walk (a fourth ring slot), so warps never wait on one another
// inside a pass.  A pass reads z and delta^i once and writes delta^{i+2} once
// (12 bytes per unknown per two sweeps); z of group k-1 stays in registers.
// The norms, the stop rule and the refinement decision follow the two-sweep
// tiled kernel (a grid barrier per pass; every block applies the stop rule to
// the fixed-order sum of the partials).
#include <math.h>

#include <algorithm>

#include "oci_device.cuh"
#include "oci_mixed_dev.cuh"

namespace oci {

namespace {

constexpr int kW2Warps = 8;  // warps per block
constexpr int kW2Threads = 32 * kW2Warps;
constexpr int kW2NP = 4;  // angles per lane
constexpr int kW2Occ = 2;  // resident blocks per SM the register allocation is built for

struct W2Args {
  int J, k0, k1;
  const int32_t *__restrict__ type;
  const float *Linv, *Cin, *Mp, *w;
  const float *__restrict__ z;
};

// Position of (cell j, first row of the lane's angles) in a tile-major array
// [J/32][4N][32]; the lane's unknown (i, p) is at +(4 i + p) * 32.
template <int N>
__device__ __forceinline__ size_t w2_base(int j, int m0) {
  return ((size_t)(j >> 5) * (4 * N) + (size_t)m0 * 4) * 32 + (j & 31);
}

// Loads of cell j for sweep i+1: z, delta^i of the cell (want_old) and its lagged
// inflow from delta^i of the upwind neighbour (zero at the slab ends, for an
// inactive lane and when delta^i is zero).
template <int N>
__device__ __forceinline__ void w2_load(float (&zr)[kW2NP][4], float (&old)[kW2NP][4], float (&uk)[kW2NP],
                                        float (&uh)[kW2NP], int j, bool act, bool want_old, bool pos, int m0, int J,
                                        bool zero, const float *__restrict__ z, const float *__restrict__ Din) {
  const size_t b = act ? w2_base<N>(j, m0) : 0;
  const float *__restrict__ zb = z + b;
  const float *__restrict__ db = Din + b;
  // upwind neighbour: j-1 for mu > 0 (previous column, or the last column of the previous tile)
  const long long off = pos ? ((j & 31) ? -1 : 31 - 4LL * N * 32) : ((j & 31) != 31 ? 1 : 4LL * N * 32 - 31);
  const bool has_in = act && !zero && (pos ? j > 0 : j < J - 1);
#pragma unroll
  for (int i = 0; i < kW2NP; i++) {
#pragma unroll
    for (int p = 0; p < 4; p++) {
      zr[i][p] = act ? zb[(i * 4 + p) * 32] : 0.f;
      old[i][p] = (act && want_old && !zero) ? db[(i * 4 + p) * 32] : 0.f;
    }
    const int rk = pos ? 1 : 0;
    uk[i] = has_in ? db[off + (i * 4 + rk) * 32] : 0.f;
    uh[i] = has_in ? db[off + (i * 4 + rk + 2) * 32] : 0.f;
  }
}

// Structured FP32 solve of the lane's four angles of its cell (one group):
// t = z + Cin u, y = sum_m w t (butterfly over the P lanes of the cell), s = Mp y,
// o = t + Linv s.  Inactive lanes give zeros and take part in the shuffles.
template <int N>
__device__ __forceinline__ void w2_solve(float (&o)[kW2NP][4], const float (&zr)[kW2NP][4], const float (&uk)[kW2NP],
                                         const float (&uh)[kW2NP], bool act, int tau, int m0, const W2Args &a) {
  constexpr int P = N / kW2NP, CW = 32 / P;
  const int tb = tau * N;
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
#pragma unroll
  for (int i = 0; i < kW2NP; i++) {
    const float4 *C4 = reinterpret_cast<const float4 *>(a.Cin + (tb + m0 + i) * 8);
    const float4 ca = C4[0], cb = C4[1];
    o[i][0] = fmaf(ca.y, uh[i], fmaf(ca.x, uk[i], zr[i][0]));
    o[i][1] = fmaf(ca.w, uh[i], fmaf(ca.z, uk[i], zr[i][1]));
    o[i][2] = fmaf(cb.y, uh[i], fmaf(cb.x, uk[i], zr[i][2]));
    o[i][3] = fmaf(cb.w, uh[i], fmaf(cb.z, uk[i], zr[i][3]));
    const float wm = a.w[m0 + i];
    y0 = fmaf(wm, o[i][0], y0);
    y1 = fmaf(wm, o[i][1], y1);
    y2 = fmaf(wm, o[i][2], y2);
    y3 = fmaf(wm, o[i][3], y3);
  }
#pragma unroll
  for (int d = CW; d < 32; d <<= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, d);
    y1 += __shfl_xor_sync(0xffffffffu, y1, d);
    y2 += __shfl_xor_sync(0xffffffffu, y2, d);
    y3 += __shfl_xor_sync(0xffffffffu, y3, d);
  }
  const float4 *M4 = reinterpret_cast<const float4 *>(a.Mp + tau * 16);
  float s[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float4 M = M4[q];
    s[q] = fmaf(M.w, y3, fmaf(M.z, y2, fmaf(M.y, y1, M.x * y0)));
  }
#pragma unroll
  for (int i = 0; i < kW2NP; i++) {
    const float4 *L4 = reinterpret_cast<const float4 *>(a.Linv + (tb + m0 + i) * 16);
#pragma unroll
    for (int p = 0; p < 4; p++) {
      const float4 L = L4[p];
      const float v = fmaf(L.w, s[3], fmaf(L.z, s[2], fmaf(L.y, s[1], fmaf(L.x, s[0], o[i][p]))));
      o[i][p] = act ? v : 0.f;
    }
  }
}

template <int N>
__device__ __forceinline__ void w2_store(float *__restrict__ Dout, int j, int m0, const float (&o)[kW2NP][4]) {
  float *__restrict__ ob = Dout + w2_base<N>(j, m0);
#pragma unroll
  for (int i = 0; i < kW2NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) ob[(i * 4 + p) * 32] = o[i][p];
}

__device__ __forceinline__ float w2_dist2(const float (&a)[kW2NP][4], const float (&b)[kW2NP][4]) {
  float e2 = 0.f;
#pragma unroll
  for (int i = 0; i < kW2NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) {
      const float d = a[i][p] - b[i][p];
      e2 = fmaf(d, d, e2);
    }
  return e2;
}

// One sweep over the warp's run (delta^i -> delta^{i+1}); the lane's sum of squared changes.
template <int N>
__device__ float w2_pass1(const W2Args &a, bool zero, const float *__restrict__ Din, float *__restrict__ Dout) {
  constexpr int P = N / kW2NP, CW = 32 / P;
  const int lane = threadIdx.x & 31, ch = lane / CW, c = lane % CW, m0 = ch * kW2NP;
  const bool pos = m0 >= N / 2;
  float e2 = 0.f;
  for (int k = a.k0; k < a.k1; k++) {
    const int j = k * CW + c;
    const bool act = j < a.J;
    const int tau = act ? a.type[j] : 0;
    float zr[kW2NP][4], old[kW2NP][4], uk[kW2NP], uh[kW2NP], o[kW2NP][4];
    w2_load<N>(zr, old, uk, uh, j, act, true, pos, m0, a.J, zero, a.z, Din);
    w2_solve<N>(o, zr, uk, uh, act, tau, m0, a);
    if (act) {
      e2 += w2_dist2(o, old);
      w2_store<N>(Dout, j, m0, o);
    }
  }
  return e2;
}

// Per-warp shared memory of the two-sweep walk: three ring slots with delta^{i+1}
// of groups k, k-1, k-2 (slot k mod 3) and one slot with delta^{i+1} of the two
// cells next to the run (left one at lanes c = CW-1, right one at lanes c = 0);
// each slot [16 unknowns of a lane][32 lanes].
constexpr int kW2Slot = kW2NP * 4 * 32;
constexpr int kW2WarpFloats = 4 * kW2Slot;

template <int N>
__device__ __forceinline__ void w2_put(float *slot, int lane, const float (&o)[kW2NP][4]) {
#pragma unroll
  for (int i = 0; i < kW2NP; i++)
#pragma unroll
    for (int p = 0; p < 4; p++) slot[(i * 4 + p) * 32 + lane] = o[i][p];
}

// One step of the two-sweep walk: delta^{i+1} of group k (z into zc, delta^{i+1}
// into its ring slot) when k < k1, then delta^{i+2} of group k-1 from zp and the
// ring when k > k0.
template <int N>
__device__ __forceinline__ void w2_step(const W2Args &a, int k, bool zero, const float *__restrict__ Din,
                                        float *__restrict__ Dout, float *ring, float (&zc)[kW2NP][4], int &tauc,
                                        const float (&zp)[kW2NP][4], int taup, float &ea, float &eb) {
  constexpr int P = N / kW2NP, CW = 32 / P;
  const int lane = threadIdx.x & 31, ch = lane / CW, c = lane % CW, m0 = ch * kW2NP;
  const bool pos = m0 >= N / 2;
  const int J = a.J;
  __syncwarp();  // the slot of group k held group k-3, read by the previous step
  if (k < a.k1) {  // sweep i+1 on group k
    const int j = k * CW + c;
    const bool act = j < J;
    tauc = act ? a.type[j] : 0;
    float old[kW2NP][4], uk[kW2NP], uh[kW2NP], o1[kW2NP][4];
    w2_load<N>(zc, old, uk, uh, j, act, true, pos, m0, J, zero, a.z, Din);
    w2_solve<N>(o1, zc, uk, uh, act, tauc, m0, a);
    if (act) ea += w2_dist2(o1, old);
    w2_put<N>(ring + (k % 3) * kW2Slot, lane, o1);
  }
  __syncwarp();
  if (k > a.k0) {  // sweep i+2 on group k-1
    const int j = (k - 1) * CW + c;
    const bool act = j < J;
    const float *prv = ring + ((k - 1) % 3) * kW2Slot;
    // upwind cell of the lane's cell: mu > 0 the cell to the left (for c = 0 the last
    // cell of group k-2, or the cell left of the run), mu < 0 the cell to the right
    // (for c = CW-1 the first cell of group k, or the cell right of the run)
    const float *edge = ring + 3 * kW2Slot;
    const float *src;
    if (pos) src = c > 0 ? prv + lane - 1 : (k - 1 > a.k0 ? ring + ((k - 2) % 3) * kW2Slot : edge) + lane + CW - 1;
    else src = c < CW - 1 ? prv + lane + 1 : (k < a.k1 ? ring + (k % 3) * kW2Slot : edge) + lane - (CW - 1);
    const bool ok = act && (pos ? j > 0 : j < J - 1);  // no inflow at the slab ends
    const int rk = pos ? 1 : 0;
    float uk[kW2NP], uh[kW2NP];
#pragma unroll
    for (int i = 0; i < kW2NP; i++) {
      uk[i] = ok ? src[(i * 4 + rk) * 32] : 0.f;
      uh[i] = ok ? src[(i * 4 + rk + 2) * 32] : 0.f;
    }
    float o2[kW2NP][4], o1[kW2NP][4];
    w2_solve<N>(o2, zp, uk, uh, act, taup, m0, a);
#pragma unroll
    for (int i = 0; i < kW2NP; i++)
#pragma unroll
      for (int p = 0; p < 4; p++) o1[i][p] = prv[(i * 4 + p) * 32 + lane];
    if (act) {
      eb += w2_dist2(o2, o1);
      w2_store<N>(Dout, j, m0, o2);
    }
  }
}

// Two sweeps over the warp's run (delta^i -> delta^{i+2}); the lane's sums of
// squared changes of both sweeps in ea, eb.  ring: the warp's kW2WarpFloats.
template <int N>
__device__ void w2_pass2(const W2Args &a, bool zero, const float *__restrict__ Din, float *__restrict__ Dout,
                         float *ring, float &ea, float &eb) {
  constexpr int P = N / kW2NP, CW = 32 / P;
  const int lane = threadIdx.x & 31, ch = lane / CW, c = lane % CW, m0 = ch * kW2NP;
  const bool pos = m0 >= N / 2;
  if (a.k0 >= a.k1) return;  // warp-uniform
  {  // delta^{i+1} of the cells next to the run: lanes c = CW-1 take cell k0 CW - 1, lanes c = 0 cell k1 CW
    const int j = c == CW - 1 ? a.k0 * CW - 1 : a.k1 * CW;
    const bool act = (c == CW - 1 || c == 0) && j >= 0 && j < a.J;
    const int tau = act ? a.type[j] : 0;
    float zr[kW2NP][4], old[kW2NP][4], uk[kW2NP], uh[kW2NP], o[kW2NP][4];
    w2_load<N>(zr, old, uk, uh, j, act, false, pos, m0, a.J, zero, a.z, Din);
    w2_solve<N>(o, zr, uk, uh, act, tau, m0, a);
    __syncwarp();  // the previous pass's reads of the edge slot are done
    w2_put<N>(ring + 3 * kW2Slot, lane, o);
  }
  float zA[kW2NP][4], zB[kW2NP][4];
  int tA = 0, tB = 0;
  // two steps per iteration with the roles of the z registers swapped (no copies)
  for (int k = a.k0; k <= a.k1; k += 2) {
    w2_step<N>(a, k, zero, Din, Dout, ring, zA, tA, zB, tB, ea, eb);
    if (k + 1 <= a.k1) w2_step<N>(a, k + 1, zero, Din, Dout, ring, zB, tB, zA, tA, ea, eb);
  }
}

template <int N, int OCC>
__global__ void __launch_bounds__(kW2Threads, OCC)
    k_mx_inner_w2(int J, int n_types, int stage, const int32_t *__restrict__ type, const float *Linv_g,
                  const float *Cin_g, const float *Mp_g, const float *w_g, const float *__restrict__ z, float *D0,
                  float *D1, DevState *ds, double *__restrict__ partials, unsigned long long *gbar, double *e_hist,
                  cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  constexpr int P = N / kW2NP, CW = 32 / P;
  extern __shared__ __align__(16) float smw[];
  __shared__ double red[kW2Warps];
  __shared__ DevState sd;
  __shared__ int s_ok, s_roll;
  unsigned long long gep = 0;  // thread 0: the arrival count the next grid barrier waits for
  const int tid = threadIdx.x, nthr = kW2Threads;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the grid
  W2Args a;
  a.J = J;
  a.type = type;
  a.z = z;
  a.Linv = Linv_g;
  a.Cin = Cin_g;
  a.Mp = Mp_g;
  a.w = w_g;
  float *ring = smw + (size_t)(tid >> 5) * kW2WarpFloats;  // this warp's ring slots
  if (stage) {
    stage_tables(smw + kW2Warps * kW2WarpFloats, n_types, N, 1, tid, nthr, a.Linv, a.Cin, a.Mp, a.w);
    __syncthreads();
  }
  const int ngr = (J + CW - 1) / CW;  // warp steps of CW cells
  const long long gw = (long long)blockIdx.x * kW2Warps + (tid >> 5), nw = (long long)gridDim.x * kW2Warps;
  a.k0 = (int)(gw * ngr / nw);
  a.k1 = (int)((gw + 1) * ngr / nw);
  bool failed = false;
  for (int sw = 0, pass = 0;; pass++) {
    const int ns = max_sweeps - sw >= 2 ? 2 : 1;
    const bool zero = sd.refine || sd.blk_i == 0;
    const float *__restrict__ Din = sd.dcur ? D1 : D0;
    float *__restrict__ Dout = sd.dcur ? D0 : D1;
    float ea = 0.f, eb = 0.f;
    if (ns == 2) w2_pass2<N>(a, zero, Din, Dout, ring, ea, eb);
    else ea = w2_pass1<N>(a, zero, Din, Dout);
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
      w2_pass1<N>(a, zero, Din, Dout);
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

size_t w2_smem(const Handle &h, bool stage) {
  return (size_t)kW2Warps * kW2WarpFloats * 4 + (stage ? mx_tables_floats(h) * 4 + 16 : 0);
}

template <int N, int OCC>
void launch_w2(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const bool stage = mx_tables_floats(h) * 4 <= 32 * 1024;
  const size_t smem = w2_smem(h, stage);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_w2<N, OCC>, kW2Threads, smem);
  constexpr int CW = 32 / (N / kW2NP);
  const int ngr = (h.J + CW - 1) / CW;
  // no block resident (per = 0) gives an empty grid: the launch is refused, the tuner skips the kernel
  const int grid = std::min(sms * per, (ngr + kW2Warps - 1) / kW2Warps);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kW2Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  k_zero_gcount<<<1, 1, 0, h.stream>>>(reinterpret_cast<unsigned long long *>(h.gbar));
  cudaLaunchKernelEx(&cfg, k_mx_inner_w2<N, OCC>, h.J, h.tt.n_types, (int)stage, (const int32_t *)h.type,
                     (const float *)h.tt.Linv32, (const float *)h.tt.Cin32, (const float *)h.tt.Mp32,
                     (const float *)h.w32, (const float *)h.z32, h.delta[0], h.delta[1], h.ds, h.partials, reinterpret_cast<unsigned long long *>(h.gbar),
                     h.e_hist, cond, use_cond, max_sweeps);
}

}  // namespace

bool mx_w2_supported(const Handle &h) { return h.G == 1 && (h.N == 8 || h.N == 16 || h.N == 32); }

void launch_w2_any(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  if (h.N == 8) launch_w2<8, kW2Occ>(h, cond, use_cond, max_sweeps);
  else if (h.N == 16) launch_w2<16, kW2Occ>(h, cond, use_cond, max_sweeps);
  else launch_w2<32, kW2Occ>(h, cond, use_cond, max_sweeps);
}

int mx_w2_set_attributes() {
  const void *ks[] = {(const void *)k_mx_inner_w2<8, kW2Occ>, (const void *)k_mx_inner_w2<16, kW2Occ>,
                      (const void *)k_mx_inner_w2<32, kW2Occ>};
  for (const void *k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kW2Warps * kW2WarpFloats * 4 + 32 * 1024 + 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(warp-run FP32 inner sweep)");
  }
  return OCI_OK;
}

}  // namespace oci
