// oci_sweep.cu -- FP64 kernels of the OCI time step (structured cell solve).
//
// Cell solve.  For cell j the OCI system (Eq. oci; multigroup Eq. fullOCIlhs)
//   (L_c - S) Psi = b,   L_c = blockdiag_{g,m} L_{c,g,m} (Eq. Aj),
//   (S Psi)_{g,m,p} = sum_{gp} dx/4 Sigma_s,gp->g phi_{gp,p},  phi_{g,p} = sum_n w_n Psi_{g,n,p}
// (Eq. scatter read with the column angle's weight) is solved exactly through
// its structure instead of a dense LU:
//   t_{g,m} = L_{g,m}^{-1} b_{g,m}
//   y_g     = sum_m w_m t_{g,m}
//   s       = Mp y,       Mp = (I - K H)^{-1} K,  H = blockdiag_g sum_m w_m L_{g,m}^{-1},
//                          K[g][gp] = dx/4 Sigma_s,gp->g I_4
//   Psi_{g,m} = t_{g,m} + L_{g,m}^{-1} s_g
// which is A_j^{-1} b_j up to rounding.  b = c + (lagged inflow) with the
// per-step constant c of Eq. rhs_sg, so t = tc + Cin u with tc = L^{-1} c
// computed once per step (k_step_const) and u the two upstream edge values.
// The register form regroups the same algebra: y = yc + sum_m (w_m Cin) u_m
// with yc = sum_m w_m tc per step (k_step_yc), and Psi_{g,m} = tc_{g,m} +
// L_{g,m}^{-1} (s_g + |mu| u placed in the inflow rows), which saves two FP64
// operations per cell, group and angle.
#include <limits.h>
#include <math.h>

#include "oci_device.cuh"

namespace oci {

// ------------------------------------------------------------------ a1
// tc_{g,m} = L_{g,m}^{-1} c_{g,m},
// c = [dx/4 Q_kL + dx/(2 v dt) psi_prev_L, dx/4 Q_kR + dx/(2 v dt) psi_prev_R, dx/4 Q_hL, dx/4 Q_hR]
__global__ void k_step_const(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                             const double *__restrict__ tdx, const double *__restrict__ v, double dt,
                             const double *__restrict__ Q, const double *__restrict__ psi_prev,
                             const double *__restrict__ Linv, double *__restrict__ tc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int gm = blockIdx.y;
  if (j >= J) return;
  const int g = gm / N;
  const int tau = type[j];
  const double dx = tdx[tau];
  const double ah = dx / (2.0 * v[g] * dt);
  double q[4] = {0.0, 0.0, 0.0, 0.0};
  if (Q) {
#pragma unroll
    for (int p = 0; p < 4; p++) q[p] = dx / 4.0 * Q[(size_t)(g * 4 + p) * Jp + j];
  }
  const double c0 = q[0] + ah * psi_prev[(size_t)(gm * 2 + 0) * Jp + j];
  const double c1 = q[1] + ah * psi_prev[(size_t)(gm * 2 + 1) * Jp + j];
  const double *L = Linv + ((size_t)tau * G * N + gm) * 16;
#pragma unroll
  for (int p = 0; p < 4; p++)
    tc[(size_t)(gm * 4 + p) * Jp + j] = L[p * 4 + 0] * c0 + L[p * 4 + 1] * c1 + L[p * 4 + 2] * q[2] + L[p * 4 + 3] * q[3];
}

// yc_{g,p} = sum_m w_m tc_{g,m,p} (ascending m), for the register sweep.
__global__ void k_step_yc(int J, int Jp, int N, const double *__restrict__ w, const double *__restrict__ tc,
                          double *__restrict__ yc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (j >= J) return;
#pragma unroll
  for (int p = 0; p < 4; p++) {
    double a = 0.0;
    for (int m = 0; m < N; m++) a = fma(w[m], tc[(size_t)((g * N + m) * 4 + p) * Jp + j], a);
    yc[(size_t)(g * 4 + p) * Jp + j] = a;
  }
}

// Deterministic block sum of one double; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) s += red[i];
  return s;
}

// ------------------------------------------------------------------ a2..a4
// One OCI sweep.  Block = CB cells x (G groups x P angle chunks); thread
// (cell, g, c) handles the angles m in [c N/P, (c+1) N/P) of group g.
// Block Jacobi (RB = false): reads Psi[cur], writes Psi[cur^1].
// Red-black (RB = true, half sweep of one colour): thread i handles cell
// 2i + colour.  PP = false: Psi[cur] is updated in place -- the neighbours have
// the other colour and are not written by this launch; one plain pointer keeps
// each cell's read of its old value before its write, which also keeps the
// loads of one angle behind the stores of the previous one.  PP = true
// (ping-pong): both colours read their own old values from Psi[cur] and write
// Psi[cur^1]; the first colour reads its neighbours from Psi[cur], the second
// from Psi[cur^1] (the first colour's new values), so no launch reads what it
// writes and the loads carry no ordering against the stores.  Same values.
// Writes this block's sum of (Psi_new - Psi_old)^2 (per colour for red-black).
// Shared memory: t [G*N*4][CB], partial y [G*P*4][CB], reduction scratch.
template <bool RB, bool PP = false>
__global__ void __launch_bounds__(256) k_oci_sweep_t(
    int J, int Jp, int N, int G, int P, int color, const int32_t *__restrict__ type,
    const double *__restrict__ Linv, const double *__restrict__ Cin, const double *__restrict__ Mp,
    const double *__restrict__ w, const double *__restrict__ inc, const double *__restrict__ tc, double *Psi0,
    double *Psi1, DevState *ds, double *__restrict__ partials, unsigned *counter, double *e_hist,
    cudaGraphConditionalHandle cond, int use_cond, int fuse, int nparts, int boff = 0, int bstride = 1) {
  extern __shared__ double sm[];
  __shared__ bool s_last;
  const int CB = blockDim.x;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P;
  const int NP = N / P, m0 = ch * NP;
  // Jacobi: logical block boff + blockIdx.x * bstride (one sweep may be split into
  // the interior blocks and the two end blocks, see launch_oci_sweep_part)
  const int lb = RB ? (int)blockIdx.x : boff + (int)blockIdx.x * bstride;
  const int j = RB ? 2 * (blockIdx.x * CB + cl) + color : lb * CB + cl;
  if (ds->done) return;  // uniform across the grid
  const int cur = ds->cur;
  constexpr bool IP = RB && !PP;  // in place
  double *Pself = cur ? Psi1 : Psi0;
  const double *__restrict__ PinJ = cur ? Psi1 : Psi0;
  double *__restrict__ PoutJ = cur ? Psi0 : Psi1;
  // upstream neighbours: the second colour of a ping-pong sweep reads the first colour's new values
  const double *__restrict__ PnbJ = (PP && color == 1) ? (cur ? Psi0 : Psi1) : PinJ;
  auto Pin = [&](size_t i) -> double { return IP ? Pself[i] : PinJ[i]; };
  auto Pnb = [&](size_t i) -> double { return IP ? Pself[i] : PnbJ[i]; };
  auto Pput = [&](size_t i, double v) {
    if (IP) Pself[i] = v;
    else PoutJ[i] = v;
  };
  double *t_s = sm;
  double *y_s = sm + (size_t)G * N * 4 * CB;
  double *red = y_s + (size_t)G * P * 4 * CB;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const int N2 = N / 2;
  const size_t tb = (size_t)tau * G * N;

  double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
  if (active) {
#pragma unroll 2
    for (int m = m0; m < m0 + NP; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      double uk, uh;
      if (m >= N2) {  // mu > 0: upstream edge is the R corner of cell j-1
        if (j > 0) {
          uk = Pnb(base + 1 * (size_t)Jp - 1);
          uh = Pnb(base + 3 * (size_t)Jp - 1);
        } else {
          uk = inc[gm * 2 + 0];
          uh = inc[gm * 2 + 1];
        }
      } else {  // mu < 0: upstream edge is the L corner of cell j+1
        if (j < J - 1) {
          uk = Pnb(base + 0 * (size_t)Jp + 1);
          uh = Pnb(base + 2 * (size_t)Jp + 1);
        } else {
          uk = inc[(G * N + gm) * 2 + 0];
          uh = inc[(G * N + gm) * 2 + 1];
        }
      }
      const double *C = Cin + (tb + gm) * 8;
      const double t0 = fma(C[1], uh, fma(C[0], uk, tc[base]));
      const double t1 = fma(C[3], uh, fma(C[2], uk, tc[base + (size_t)Jp]));
      const double t2 = fma(C[5], uh, fma(C[4], uk, tc[base + 2 * (size_t)Jp]));
      const double t3 = fma(C[7], uh, fma(C[6], uk, tc[base + 3 * (size_t)Jp]));
      double *ts = t_s + (size_t)(gm * 4) * CB + cl;
      ts[0] = t0;
      ts[CB] = t1;
      ts[2 * CB] = t2;
      ts[3 * CB] = t3;
      const double wm = w[m];
      y0 = fma(wm, t0, y0);
      y1 = fma(wm, t1, y1);
      y2 = fma(wm, t2, y2);
      y3 = fma(wm, t3, y3);
    }
    double *ys = y_s + (size_t)(gy * 4) * CB + cl;
    ys[0] = y0;
    ys[CB] = y1;
    ys[2 * CB] = y2;
    ys[3 * CB] = y3;
  }
  __syncthreads();
  double e2 = 0.0;
  if (active) {
    // s_g = sum_{gp} Mp[g][gp] y_gp,  y_gp = sum over the gp chunks (fixed order)
    const int G4 = 4 * G;
    const double *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int k = 0; k < G4; k++) {
      const int gp = k >> 2, q = k & 3;
      double yk = y_s[(size_t)((gp * P) * 4 + q) * CB + cl];
      for (int c = 1; c < P; c++) yk += y_s[(size_t)((gp * P + c) * 4 + q) * CB + cl];
      s0 = fma(M[k], yk, s0);
      s1 = fma(M[G4 + k], yk, s1);
      s2 = fma(M[2 * G4 + k], yk, s2);
      s3 = fma(M[3 * G4 + k], yk, s3);
    }
#pragma unroll 2
    for (int m = m0; m < m0 + NP; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const double *L = Linv + (tb + gm) * 16;
      const double *ts = t_s + (size_t)(gm * 4) * CB + cl;
      double o[4];
#pragma unroll
      for (int p = 0; p < 4; p++)
        o[p] = fma(L[p * 4 + 3], s3, fma(L[p * 4 + 2], s2, fma(L[p * 4 + 1], s1, fma(L[p * 4 + 0], s0, ts[p * CB]))));
      double old[4];
#pragma unroll
      for (int p = 0; p < 4; p++) old[p] = Pin(base + (size_t)p * Jp);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const double d = o[p] - old[p];
        e2 = fma(d, d, e2);
        Pput(base + (size_t)p * Jp, o[p]);
      }
    }
  }
  const double bs = block_sum(e2, red);
  const int slot = lb + (RB ? color * gridDim.x : 0);
  if (!fuse) {
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[slot] = bs;
    return;
  }
  // the block that finishes last reduces all partials and applies the stop rule
  if (publish_partial(partials, slot, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, nparts, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      *counter = 0;
      finish_fp64(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

const void *k_oci_sweep_ptr() { return (const void *)k_oci_sweep_t<false>; }
const void *k_oci_sweep_rb_ptr() { return (const void *)k_oci_sweep_t<true>; }
const void *k_oci_sweep_rbpp_ptr() { return (const void *)k_oci_sweep_t<true, true>; }

size_t sweep_smem(int N, int G, int cb, int P, size_t es) {
  return (size_t)cb * ((size_t)G * N * 4 + (size_t)G * P * 4) * es + 64 * sizeof(double);
}

// Default launch shape (used when the autotuner is off): the largest block of
// cells that keeps <= 256 threads and <= 96 KB of shared memory, one chunk.
// One plain Jacobi sweep out = A^{-1}(c + B in) with the given per-step constant
// (tc = A^{-1}-premultiplied c) and incident flux, on arbitrary buffers: the
// operator apply of the Krylov acceleration (no norm, no stop rule; ds_apply
// is a device state with cur = 0 and done = 0, read only).
void launch_oci_apply(Handle &h, const double *in, double *out, const double *tc, const double *inc,
                      DevState *ds_apply) {
  SweepCfg c = sweep_config(h);
  dim3 block(c.cells_per_block, h.G * c.chunks);
  cudaGraphConditionalHandle none{};
  k_oci_sweep_t<false><<<c.grid, block, c.smem, h.stream>>>(h.J, h.Jp, h.N, h.G, c.chunks, -1, h.type, h.tt.Linv,
                                                            h.tt.Cin, h.tt.Mp, h.w, inc, tc, const_cast<double *>(in),
                                                            out, ds_apply, h.partials, h.counter, nullptr, none, 0, 0,
                                                            c.grid);
}

SweepCfg sweep_config(const Handle &h) {
  SweepCfg c;
  int cb = h.tune_cb, P = h.tune_P;
  if (cb <= 0) {
    P = 1;
    cb = 128;
    while (cb > 1 && ((size_t)cb * h.G > 256 || sweep_smem(h.N, h.G, cb, 1, 8) > 96 * 1024)) cb /= 2;
  }
  c.cells_per_block = cb;
  c.chunks = P;
  c.grid = (h.J + cb - 1) / cb;
  c.smem = sweep_smem(h.N, h.G, cb, P, 8);
  return c;
}

void launch_step_const(Handle &h) {
  dim3 grid((h.J + 255) / 256, h.G * h.N);
  k_step_const<<<grid, 256, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.dx, h.v, h.dt, h.Q, h.psi_prev,
                                           h.tt.Linv, h.tc);
  k_step_yc<<<dim3((h.J + 255) / 256, h.G), 256, 0, h.stream>>>(h.J, h.Jp, h.N, h.w, h.tc, h.yc);
}

// Loads of the iterate: plain, or through L2 only (ld.global.cg) where another
// block of the same launch may have rewritten the line since this SM cached it.
template <bool CG>
__device__ __forceinline__ double ld_psi(const double *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// The inflows u of thread (cl, gy) of cell j, as reg_cells<NP, true> reads them
// (through L2): the upstream corners of the neighbour in Pin, or the incident
// flux at the slab ends; zeros for an inactive cell.
template <int NP>
__device__ __forceinline__ void reg_inflows(int j, int J, int Jp, int N, int G, int gy, const double *__restrict__ inc,
                                            const double *Pin, double (&u)[NP][2]) {
  const int P = N / NP, g = gy / P, m0 = (gy % P) * NP, N2 = N / 2;
  const bool active = j < J;
#pragma unroll
  for (int i = 0; i < NP; i++) {
    const int m = m0 + i, gm = g * N + m;
    const size_t base = (size_t)gm * 4 * Jp + j;
    double uk = 0.0, uh = 0.0;
    if (active) {
      if (m >= N2) {
        if (j > 0) {
          uk = __ldcg(Pin + base + (size_t)Jp - 1);
          uh = __ldcg(Pin + base + 3 * (size_t)Jp - 1);
        } else {
          uk = inc[gm * 2 + 0];
          uh = inc[gm * 2 + 1];
        }
      } else if (j < J - 1) {
        uk = __ldcg(Pin + base + 1);
        uh = __ldcg(Pin + base + 2 * (size_t)Jp + 1);
      } else {
        uk = inc[(G * N + gm) * 2 + 0];
        uh = inc[(G * N + gm) * 2 + 1];
      }
    }
    u[i][0] = uk;
    u[i][1] = uh;
  }
}

// The cells of one block of the register form: thread (cl, gy) of cell j; the
// block's shared memory holds y [G*P*4][CB], y reduced [4G][CB] and s [4G][CB].
// Writes Pout for the active cells and returns the thread's sum of
// (Psi_new - Psi_old)^2.  Contains block-wide barriers: every thread calls it.
// HOIST: the cell's inflow weights, L^{-1}, step constant and |mu| of the
// thread's angles come from the caller's registers (Wh, Lh, tch, amh) instead
// of memory.  PRE: the inflows u were loaded by the caller (upre, reg_inflows).
template <int NP, bool CG, bool HOIST = false, bool PRE = false>
__device__ __forceinline__ double reg_cells(int j, int J, int Jp, int N, int G, int CB, int cl, int gy,
                                            const int32_t *__restrict__ type, const double *__restrict__ Linv,
                                            const double *__restrict__ Mp, const double *__restrict__ inc,
                                            const double *__restrict__ tc, const double *__restrict__ Pin,
                                            double *__restrict__ Pout, const double *__restrict__ Pnb,
                                            const double *__restrict__ Win, const double *__restrict__ yc,
                                            const double *__restrict__ mu, double *y_s, double *yr_s, double *s_s,
                                            const double (*Wh)[8] = nullptr, const double (*Lh)[16] = nullptr,
                                            const double (*tch)[4] = nullptr, const double *amh = nullptr,
                                            const double (*upre)[2] = nullptr) {
  const int P = N / NP, G4 = 4 * G;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const int N2 = N / 2;
  const size_t tb = (size_t)tau * G * N;
  double u[NP][2];
  // CG (all sweeps in one launch): the old values are loaded with the inflows,
  // so one round trip to L2 per sweep serves both; the one-sweep kernel loads
  // them where they are used
  double old[CG ? NP : 1][4];
  double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
  if (active) {
    if constexpr (CG) {
#pragma unroll
      for (int i = 0; i < NP; i++)
#pragma unroll
        for (int p = 0; p < 4; p++) old[i][p] = __ldcg(Pin + (size_t)(g * N + m0 + i) * 4 * Jp + j + (size_t)p * Jp);
    }
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      double uk, uh;
      if constexpr (PRE) {
        uk = upre[i][0];
        uh = upre[i][1];
      } else if (m >= N2) {
        if (j > 0) {
          uk = ld_psi<CG>(Pnb + base + (size_t)Jp - 1);
          uh = ld_psi<CG>(Pnb + base + 3 * (size_t)Jp - 1);
        } else {
          uk = inc[gm * 2 + 0];
          uh = inc[gm * 2 + 1];
        }
      } else if (j < J - 1) {
        uk = ld_psi<CG>(Pnb + base + 1);
        uh = ld_psi<CG>(Pnb + base + 2 * (size_t)Jp + 1);
      } else {
        uk = inc[(G * N + gm) * 2 + 0];
        uh = inc[(G * N + gm) * 2 + 1];
      }
      u[i][0] = uk;
      u[i][1] = uh;
      const double *W;
      if constexpr (HOIST) W = Wh[i];
      else W = Win + (tb + gm) * 8;
      y0 = fma(W[1], uh, fma(W[0], uk, y0));
      y1 = fma(W[3], uh, fma(W[2], uk, y1));
      y2 = fma(W[5], uh, fma(W[4], uk, y2));
      y3 = fma(W[7], uh, fma(W[6], uk, y3));
    }
  }
  {
    double *ys = y_s + (size_t)(gy * 4) * CB + cl;
    ys[0] = y0;
    ys[CB] = y1;
    ys[2 * CB] = y2;
    ys[3 * CB] = y3;
  }
  __syncthreads();
  for (int q = ch; q < 4; q += P) {  // y_{g,q} = yc + fixed-order sum over the group's chunks
    double v = active ? yc[(size_t)(g * 4 + q) * Jp + j] : 0.0;
    for (int k = 0; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * CB + cl];
    yr_s[(size_t)(g * 4 + q) * CB + cl] = v;
  }
  __syncthreads();
  if (active)
    for (int q = ch; q < 4; q += P) {  // s_{g,q} = sum_k Mp[g*4+q][k] y_k
      const double *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
      double v = 0.0;
      for (int k = 0; k < G4; k++) v = fma(M[k], yr_s[(size_t)k * CB + cl], v);
      s_s[(size_t)(g * 4 + q) * CB + cl] = v;
    }
  __syncthreads();
  double e2 = 0.0;
  if (active) {
    const double s0 = s_s[(size_t)(g * 4 + 0) * CB + cl], s1 = s_s[(size_t)(g * 4 + 1) * CB + cl];
    const double s2 = s_s[(size_t)(g * 4 + 2) * CB + cl], s3 = s_s[(size_t)(g * 4 + 3) * CB + cl];
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int m = m0 + i;
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const double *L;
      double am;  // v = s + |mu| u in the rows the inflow feeds (0, 2 for mu > 0; 1, 3 for mu < 0)
      if constexpr (HOIST) {
        L = Lh[i];
        am = amh[i];
      } else {
        L = Linv + (tb + gm) * 16;
        am = fabs(mu[m]);
      }
      const bool pos = m >= N2;
      const double v0 = pos ? fma(am, u[i][0], s0) : s0, v1 = pos ? s1 : fma(am, u[i][0], s1);
      const double v2 = pos ? fma(am, u[i][1], s2) : s2, v3 = pos ? s3 : fma(am, u[i][1], s3);
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const double o = fma(L[p * 4 + 3], v3, fma(L[p * 4 + 2], v2, fma(L[p * 4 + 1], v1, fma(L[p * 4 + 0], v0, HOIST ? tch[HOIST ? i : 0][p] : tc[base + (size_t)p * Jp]))));
        const double d = o - (CG ? old[CG ? i : 0][p] : Pin[base + (size_t)p * Jp]);
        e2 = fma(d, d, e2);
        Pout[base + (size_t)p * Jp] = o;
      }
    }
  }
  return e2;
}

// ---------------------------------------------------------------- register form (FP64)
// The same FP64 sweep with the N angles of a cell split over P = N/NP threads,
// each keeping its NP angles' inflow u in registers: no per-angle staging in
// shared memory, so problems with many unknowns per cell (large N*G) keep more
// warps resident.  y = yc + sum_m Win_m u_m is reduced over the chunks in a
// fixed order, s = Mp y is split over the chunk threads of each group, and
// Psi = tc + Linv (s + |mu| u in the inflow rows).  Cin and w are not read here
// (Win = w Cin and yc carry them); they stay in the argument list the staged
// form shares.  The norm
// and stop rule are fused into the last block.  RB = false: Jacobi ordering.
// RB = true: half sweep of one colour (cell j = 2i + colour) on ping-pong
// buffers as in k_oci_sweep_t<true, true>; the first colour only writes its
// block partials, the second reduces both colours' (nparts in all).
template <int NP, bool RB = false>
__global__ void __launch_bounds__(256) k_oci_sweep_reg(
    int J, int Jp, int N, int G, const int32_t *__restrict__ type, const double *__restrict__ Linv,
    const double *__restrict__ Cin, const double *__restrict__ Mp, const double *__restrict__ w,
    const double *__restrict__ inc, const double *__restrict__ tc, double *Psi0, double *Psi1, DevState *ds,
    double *__restrict__ partials, unsigned *counter, double *e_hist, cudaGraphConditionalHandle cond, int use_cond,
    int color, int nparts, const double *__restrict__ Win, const double *__restrict__ yc,
    const double *__restrict__ mu, int fuse = 1, int boff = 0, int bstride = 1) {
  extern __shared__ double smrd[];
  __shared__ double red[8];
  __shared__ bool s_last;
  const int CB = blockDim.x, P = N / NP;
  const int cl = threadIdx.x, gy = threadIdx.y;
  // Jacobi: logical block boff + blockIdx.x * bstride (as in k_oci_sweep_t)
  const int lb = RB ? (int)blockIdx.x : boff + (int)blockIdx.x * bstride;
  const int j = RB ? 2 * (blockIdx.x * CB + cl) + color : lb * CB + cl;
  const int tid = threadIdx.y * CB + threadIdx.x;
  if (ds->done) return;  // uniform across the grid
  const int cur = ds->cur;
  const double *__restrict__ Pin = cur ? Psi1 : Psi0;
  double *__restrict__ Pout = cur ? Psi0 : Psi1;
  // upstream neighbours: the second colour of a red-black sweep reads the first colour's new values
  const double *__restrict__ Pnb = (RB && color == 1) ? (cur ? Psi0 : Psi1) : Pin;
  double *y_s = smrd;                           // [G*P*4][CB]
  double *yr_s = y_s + (size_t)G * P * 4 * CB;  // [4G][CB]
  double *s_s = yr_s + (size_t)4 * G * CB;      // [4G][CB]
  const double e2 = reg_cells<NP, false>(j, J, Jp, N, G, CB, cl, gy, type, Linv, Mp, inc, tc, Pin, Pout, Pnb, Win,
                                         yc, mu, y_s, yr_s, s_s);
  const double bs = block_sum(e2, red);
  const int slot = lb + (RB ? color * gridDim.x : 0);
  if ((RB && color == 0) || !fuse) {
    if (tid == 0) partials[slot] = bs;
    return;
  }
  if (publish_partial(partials, slot, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, nparts, red);
    if (tid == 0) {
      *counter = 0;
      finish_fp64(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
  (void)Cin;
  (void)w;
}

// ---------------------------------------------------------------- register form, all sweeps in one launch
// A problem whose cell blocks are all resident at once spends most of a sweep
// on the launch.  This kernel runs the consecutive Jacobi sweeps of a step in
// one cooperative launch, one block per cell block: each block sweeps its
// cells, writes its partial, meets the others at a grid barrier (bounded spin)
// and sums all nb partials in the fixed order of the one-sweep kernel's last
// block, so every block takes the same stop-rule decision on its own copy of
// the device state and the iterates, norms and sweep counts are those of one
// launch per sweep, bit for bit.  Partials are double-buffered by sweep parity
// (a block that starts the next sweep cannot overwrite values another block is
// still summing); the iterate is read through L2, since this SM's L1 may hold
// lines that other blocks rewrote in the previous sweep.  The launch ends when
// the step is done or after max_sweeps sweeps; a barrier that gives up records
// OCI_E_TIMEOUT and ends the step.  gcount is zero at the launch.
template <int NP>
__global__ void __launch_bounds__(256, 1) k_oci_sweep_reg_ms(
    int J, int Jp, int N, int G, const int32_t *__restrict__ type, const double *__restrict__ Linv,
    const double *__restrict__ Mp, const double *__restrict__ inc, const double *__restrict__ tc, double *Psi0,
    double *Psi1, DevState *ds, double *__restrict__ partials, unsigned long long *gcount, double *e_hist,
    cudaGraphConditionalHandle cond, int use_cond, const double *__restrict__ Win, const double *__restrict__ yc,
    const double *__restrict__ mu, int max_sweeps) {
  extern __shared__ double smrd[];
  __shared__ double red[8];
  __shared__ DevState sd;
  __shared__ int s_ok;
  const int CB = blockDim.x, P = N / NP;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int tid = threadIdx.y * CB + threadIdx.x;
  const int nb = gridDim.x;
  const int j = blockIdx.x * CB + cl;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the grid
  double *y_s = smrd;
  double *yr_s = y_s + (size_t)G * P * 4 * CB;
  double *s_s = yr_s + (size_t)4 * G * CB;
  // with two angles per thread the cell's constants stay in registers across the sweeps
  // (the grid barrier's fences would otherwise have them reloaded in every sweep)
  constexpr bool HOIST = NP == 2;
  constexpr int NH = HOIST ? NP : 1;
  double Wr[NH][8], Lr[NH][16], tcr[NH][4], amr[NH];
  if constexpr (HOIST) {
    const bool active = j < J;
    const size_t tb = (size_t)(active ? type[j] : 0) * G * N;
    const int g = gy / P, m0 = (gy % P) * NP;
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int gm = g * N + m0 + i;
      const size_t base = (size_t)gm * 4 * Jp + j;
#pragma unroll
      for (int k = 0; k < 8; k++) Wr[i][k] = active ? Win[(tb + gm) * 8 + k] : 0.0;
#pragma unroll
      for (int k = 0; k < 16; k++) Lr[i][k] = active ? Linv[(tb + gm) * 16 + k] : 0.0;
#pragma unroll
      for (int p = 0; p < 4; p++) tcr[i][p] = active ? tc[base + (size_t)p * Jp] : 0.0;
      amr[i] = fabs(mu[m0 + i]);
    }
  }
  bool failed = false;
  // the inflows of a sweep are loaded right after the previous sweep's grid barrier,
  // before its norm and stop rule (they do not depend on the decision)
  double u[NP][2];
  reg_inflows<NP>(j, J, Jp, N, G, gy, inc, sd.cur ? Psi1 : Psi0, u);
  for (int sw = 0;; sw++) {
    const int cur = sd.cur;
    const double *Pin = cur ? Psi1 : Psi0;
    double *Pout = cur ? Psi0 : Psi1;
    const double e2 = reg_cells<NP, true, HOIST, true>(j, J, Jp, N, G, CB, cl, gy, type, Linv, Mp, inc, tc, Pin,
                                                       Pout, Pin, Win, yc, mu, y_s, yr_s, s_s, Wr, Lr, tcr, amr, u);
    const double bs = block_sum(e2, red);
    double *part = partials + (size_t)(sw & 1) * nb;
    if (tid == 0) {
      part[blockIdx.x] = bs;
      s_ok = grid_barrier_count(gcount, (unsigned long long)(sw + 1) * nb, sd.spin);
    }
    __syncthreads();
    if (!s_ok) {
      failed = true;
      break;
    }
    reg_inflows<NP>(j, J, Jp, N, G, gy, inc, Pout, u);  // the next sweep's (harmless if the step ends here)
    const double tot = block_sum_fixed(part, nb, red);
    if (tid == 0) finish_fp64(&sd, blockIdx.x == 0 ? e_hist : nullptr, sqrt(tot), cond, 0);
    __syncthreads();
    if (sd.done || sw + 1 >= max_sweeps) break;  // uniform: every block holds the same state
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (failed) {
      sd.status = OCI_E_TIMEOUT;
      sd.done = 1;
    }
    *ds = sd;
    if (use_cond && sd.done) cudaGraphSetConditional(cond, 0);
  }
}

// ---------------------------------------------------------------- register form, one cluster, iterate on chip
// A problem of at most 16 cell blocks runs all sweeps of a step in one thread-
// block cluster, one block per cell block, with the iterate held on chip: each
// thread keeps its NP angles' four corner values of its cell in registers from
// sweep to sweep, and only the values a neighbouring cell reads (the two
// downstream corners of each angle) are published in shared memory, double-
// buffered by sweep parity.  A cell reads its upstream neighbour there (its
// own block's buffer, or through distributed shared memory the adjacent
// block's at the block's first and last cell), block partials of the norm are
// read from every block's shared memory the same way, and one hardware cluster
// barrier per sweep orders it all: no global-memory round trip per sweep and
// no spin.  The arithmetic and the partial sums are those of k_oci_sweep_reg
// with the same shape (same operations in the same order), so the iterates,
// norms and sweep counts are those of one launch per sweep, bit for bit.  The
// last iterate goes to Psi[cur] when the launch ends (the step is done, or
// max_sweeps sweeps); Psi[cur^1], which the next sweep only writes, is not
// touched.
__device__ __forceinline__ double ld_cluster(const double *local, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(r) : "memory");
  return v;
}

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int NP>
__global__ void __launch_bounds__(256, 1) k_oci_sweep_cl(
    int J, int Jp, int N, int G, const int32_t *__restrict__ type, const double *__restrict__ Linv,
    const double *__restrict__ Mp, const double *__restrict__ inc, const double *__restrict__ tc, double *Psi0,
    double *Psi1, DevState *ds, double *e_hist, cudaGraphConditionalHandle cond, int use_cond,
    const double *__restrict__ Win, const double *__restrict__ yc, const double *__restrict__ mu, int max_sweeps) {
  extern __shared__ double smrd[];
  __shared__ double red[8];
  __shared__ double part[2];
  __shared__ DevState sd;
  const int CB = blockDim.x, P = N / NP, G4 = 4 * G, GP = G * P;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P, m0 = ch * NP;
  const int tid = threadIdx.y * CB + threadIdx.x;
  const int nthr = CB * blockDim.y;
  const unsigned lb = blockIdx.x, nb = gridDim.x;  // the grid is one cluster
  const int j = (int)lb * CB + cl;
  const int N2 = N / 2;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const size_t tb = (size_t)tau * G * N;
  if (tid == 0) sd = *ds;
  __syncthreads();
  if (sd.done) return;  // uniform across the cluster
  double *y_s = smrd;                           // [G*P*4][CB]
  double *yr_s = y_s + (size_t)G * P * 4 * CB;  // [4G][CB]
  double *s_s = yr_s + (size_t)G4 * CB;         // [4G][CB]
  double *E = s_s + (size_t)G4 * CB;            // [2][G*P][NP][2][CB] published downstream corners
  auto eix = [&](int par, int i, int k, int c) -> size_t {
    return ((((size_t)par * GP + gy) * NP + i) * 2 + k) * CB + c;
  };
  double ps[NP][4];
  {
    const double *Pin = sd.cur ? Psi1 : Psi0;
#pragma unroll
    for (int i = 0; i < NP; i++)
#pragma unroll
      for (int p = 0; p < 4; p++) ps[i][p] = active ? Pin[(size_t)((g * N + m0 + i) * 4 + p) * Jp + j] : 0.0;
  }
  // The cell's constants of the solve -- the inflow weights, L^{-1}, the step constant
  // and |mu| of the thread's angles -- are the same in every sweep; with two angles
  // per thread they stay in registers (the cluster barrier's memory clobber would
  // otherwise have them reloaded in every sweep).
  constexpr bool HOIST = NP == 2;
  constexpr int NH = HOIST ? NP : 1;
  double Wr[NH][8], Lr[NH][16], tcr[NH][4], amr[NH];
  if constexpr (HOIST) {
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const int gm = g * N + m0 + i;
      const size_t base = (size_t)gm * 4 * Jp + j;
#pragma unroll
      for (int k = 0; k < 8; k++) Wr[i][k] = active ? Win[(tb + gm) * 8 + k] : 0.0;
#pragma unroll
      for (int k = 0; k < 16; k++) Lr[i][k] = active ? Linv[(tb + gm) * 16 + k] : 0.0;
#pragma unroll
      for (int p = 0; p < 4; p++) tcr[i][p] = active ? tc[base + (size_t)p * Jp] : 0.0;
      amr[i] = fabs(mu[m0 + i]);
    }
  }
  auto publish = [&](int par) {
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const bool pos = m0 + i >= N2;  // mu > 0: the right corners feed cell j+1, else the left ones cell j-1
      E[eix(par, i, 0, cl)] = pos ? ps[i][1] : ps[i][0];
      E[eix(par, i, 1, cl)] = pos ? ps[i][3] : ps[i][2];
    }
  };
  publish(0);
  cluster_barrier();
  for (int sw = 0;; sw++) {
    const int par = sw & 1;
    double u[NP][2];
    double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const int m = m0 + i;
        const int gm = g * N + m;
        double uk, uh;
        if (m >= N2) {
          if (j == 0) {
            uk = inc[gm * 2 + 0];
            uh = inc[gm * 2 + 1];
          } else if (cl > 0) {
            uk = E[eix(par, i, 0, cl - 1)];
            uh = E[eix(par, i, 1, cl - 1)];
          } else {
            uk = ld_cluster(E + eix(par, i, 0, CB - 1), lb - 1);
            uh = ld_cluster(E + eix(par, i, 1, CB - 1), lb - 1);
          }
        } else if (j == J - 1) {
          uk = inc[(G * N + gm) * 2 + 0];
          uh = inc[(G * N + gm) * 2 + 1];
        } else if (cl < CB - 1) {
          uk = E[eix(par, i, 0, cl + 1)];
          uh = E[eix(par, i, 1, cl + 1)];
        } else {
          uk = ld_cluster(E + eix(par, i, 0, 0), lb + 1);
          uh = ld_cluster(E + eix(par, i, 1, 0), lb + 1);
        }
        u[i][0] = uk;
        u[i][1] = uh;
        double W[8];
#pragma unroll
        for (int k = 0; k < 8; k++) W[k] = HOIST ? Wr[HOIST ? i : 0][k] : Win[(tb + gm) * 8 + k];
        y0 = fma(W[1], uh, fma(W[0], uk, y0));
        y1 = fma(W[3], uh, fma(W[2], uk, y1));
        y2 = fma(W[5], uh, fma(W[4], uk, y2));
        y3 = fma(W[7], uh, fma(W[6], uk, y3));
      }
    }
    {
      double *ys = y_s + (size_t)(gy * 4) * CB + cl;
      ys[0] = y0;
      ys[CB] = y1;
      ys[2 * CB] = y2;
      ys[3 * CB] = y3;
    }
    __syncthreads();
    for (int q = ch; q < 4; q += P) {
      double v = active ? yc[(size_t)(g * 4 + q) * Jp + j] : 0.0;
      for (int k = 0; k < P; k++) v += y_s[(size_t)((g * P + k) * 4 + q) * CB + cl];
      yr_s[(size_t)(g * 4 + q) * CB + cl] = v;
    }
    __syncthreads();
    if (active)
      for (int q = ch; q < 4; q += P) {
        const double *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4 + q) * G4;
        double v = 0.0;
        for (int k = 0; k < G4; k++) v = fma(M[k], yr_s[(size_t)k * CB + cl], v);
        s_s[(size_t)(g * 4 + q) * CB + cl] = v;
      }
    __syncthreads();
    double e2 = 0.0;
    if (active) {
      const double s0 = s_s[(size_t)(g * 4 + 0) * CB + cl], s1 = s_s[(size_t)(g * 4 + 1) * CB + cl];
      const double s2 = s_s[(size_t)(g * 4 + 2) * CB + cl], s3 = s_s[(size_t)(g * 4 + 3) * CB + cl];
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const int m = m0 + i;
        const int gm = g * N + m;
        const size_t base = (size_t)gm * 4 * Jp + j;
        double L[16], tcv[4];
#pragma unroll
        for (int k = 0; k < 16; k++) L[k] = HOIST ? Lr[HOIST ? i : 0][k] : Linv[(tb + gm) * 16 + k];
#pragma unroll
        for (int p = 0; p < 4; p++) tcv[p] = HOIST ? tcr[HOIST ? i : 0][p] : tc[base + (size_t)p * Jp];
        const double am = HOIST ? amr[HOIST ? i : 0] : fabs(mu[m]);
        const bool pos = m >= N2;
        const double v0 = pos ? fma(am, u[i][0], s0) : s0, v1 = pos ? s1 : fma(am, u[i][0], s1);
        const double v2 = pos ? fma(am, u[i][1], s2) : s2, v3 = pos ? s3 : fma(am, u[i][1], s3);
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const double o = fma(L[p * 4 + 3], v3, fma(L[p * 4 + 2], v2, fma(L[p * 4 + 1], v1, fma(L[p * 4 + 0], v0, tcv[p]))));
          const double d = o - ps[i][p];
          e2 = fma(d, d, e2);
          ps[i][p] = o;
        }
      }
    }
    publish(par ^ 1);
    const double bs = block_sum(e2, red);
    if (tid == 0) part[par] = bs;
    cluster_barrier();  // the new corners and every block's partial are visible cluster-wide
    // fixed-order sum of the nb block partials, as the one-sweep kernel's last block does
    double s = 0.0;
    for (int i = tid; i < (int)nb; i += nthr) s += ld_cluster(&part[par], (unsigned)i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (nthr + 31) / 32; w++) t += red[w];
      finish_fp64(&sd, lb == 0 ? e_hist : nullptr, sqrt(t), cond, 0);
    }
    __syncthreads();
    if (sd.done || sw + 1 >= max_sweeps) break;  // uniform: every block holds the same state
  }
  // the last iterate to Psi[cur] (the stop rule flipped cur with every sweep)
  if (active) {
    double *Pnew = sd.cur ? Psi1 : Psi0;
#pragma unroll
    for (int i = 0; i < NP; i++)
#pragma unroll
      for (int p = 0; p < 4; p++) Pnew[(size_t)((g * N + m0 + i) * 4 + p) * Jp + j] = ps[i][p];
  }
  if (lb == 0 && tid == 0) {
    *ds = sd;
    if (use_cond && sd.done) cudaGraphSetConditional(cond, 0);
  }
  cluster_barrier();  // no block leaves while another may still read its shared memory
}

size_t sweep_reg_smem(int G, int cb, int P) { return (size_t)cb * ((size_t)G * P * 4 + 8 * (size_t)G) * 8; }

const void *k_oci_sweep_reg_ptr(int np) {
  return np == 2 ? (const void *)k_oci_sweep_reg<2> : np == 4 ? (const void *)k_oci_sweep_reg<4>
                                                               : (const void *)k_oci_sweep_reg<8>;
}

// Grid of k_oci_sweep_reg_ms for the current register shape: the number of
// cell blocks when all of them can be resident at once (and two sets of their
// partials fit the reduction scratch), else 0 -- one launch per sweep.
// OCI_SWEEP_MS=0 keeps one launch per sweep.
int sweep_ms_grid(const Handle &h) {
  if (!h.tune_reg || h.ordering == OCI_ORDER_RED_BLACK || h.precision != OCI_FP64 ||
      h.solver == OCI_SOLVER_DENSE_LU)
    return 0;
  const char *v = hook_env("OCI_SWEEP_MS");
  if (v && v[0] == '0') return 0;
  const int cb = h.tune_cb, P = h.tune_P, np = h.N / P;
  const int nb = (h.J + cb - 1) / cb;
  if (2 * nb > h.n_partials) return 0;
  const void *k = np == 2 ? (const void *)k_oci_sweep_reg_ms<2>
                  : np == 4 ? (const void *)k_oci_sweep_reg_ms<4>
                            : (const void *)k_oci_sweep_reg_ms<8>;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, cb * h.G * P, sweep_reg_smem(h.G, cb, P)) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb <= sms * per ? nb : 0;
}

// Up to max_sweeps sweeps of the step in one cooperative launch (grid from
// sweep_ms_grid); ends earlier when the step is done.  Outside a graph the
// barrier count is zeroed first.
void launch_oci_sweep_ms(Handle &h, int grid, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const int cb = h.tune_cb, P = h.tune_P, np = h.N / P;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(cb, h.G * P);
  cfg.dynamicSmemBytes = sweep_reg_smem(h.G, cb, P);
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the two words of the barrier record as one count; in the graph it was zeroed
  // at the start of the step and the one launch runs to the step's end
  unsigned long long *gcount = reinterpret_cast<unsigned long long *>(h.gbar);
  if (!use_cond) cudaMemsetAsync(gcount, 0, sizeof(unsigned long long), h.stream);
#define OCI_SWEEP_MS(NP)                                                                                          \
  cudaLaunchKernelEx(&cfg, k_oci_sweep_reg_ms<NP>, h.J, h.Jp, h.N, h.G, (const int32_t *)h.type,                 \
                     (const double *)h.tt.Linv, (const double *)h.tt.Mp, (const double *)h.inc,                 \
                     (const double *)h.tc, h.Psi[0], h.Psi[1], h.ds, h.partials, gcount, h.e_hist, cond, use_cond, \
                     (const double *)h.tt.Win, (const double *)h.yc, (const double *)h.mu, max_sweeps)
  if (np == 2) OCI_SWEEP_MS(2);
  else if (np == 4) OCI_SWEEP_MS(4);
  else OCI_SWEEP_MS(8);
#undef OCI_SWEEP_MS
}

// Shared memory of k_oci_sweep_cl: the register form's plus the published
// corners, [2][G*P][NP][2][CB] doubles.
static size_t sweep_cl_smem(int N, int G, int cb, int P) {
  return sweep_reg_smem(G, cb, P) + (size_t)2 * G * N * 2 * cb * 8;
}

static const void *k_oci_sweep_cl_ptr(int np) {
  return np == 2 ? (const void *)k_oci_sweep_cl<2> : np == 4 ? (const void *)k_oci_sweep_cl<4>
                                                              : (const void *)k_oci_sweep_cl<8>;
}

// Cluster launch of k_oci_sweep_cl over nb blocks (the whole grid one cluster).
static void sweep_cl_config(const Handle &h, int nb, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr) {
  const int cb = h.tune_cb, P = h.tune_P;
  cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(cb, h.G * P);
  cfg.dynamicSmemBytes = sweep_cl_smem(h.N, h.G, cb, P);
  cfg.stream = h.stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nb;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

// Blocks of k_oci_sweep_cl for the current register shape: the number of cell
// blocks when there are at most 16 and one cluster of them can be scheduled on
// this GPU, else 0.  OCI_SWEEP_MS=0 or =grid turns the cluster form off.
int sweep_cl_grid(const Handle &h) {
  if (!h.tune_reg || h.ordering == OCI_ORDER_RED_BLACK || h.precision != OCI_FP64 ||
      h.solver == OCI_SOLVER_DENSE_LU)
    return 0;
  const char *v = hook_env("OCI_SWEEP_MS");
  if (v && (v[0] == '0' || v[0] == 'g')) return 0;
  const int cb = h.tune_cb, P = h.tune_P, np = h.N / P;
  const int nb = (h.J + cb - 1) / cb;
  if (nb > 16) return 0;
  const void *k = k_oci_sweep_cl_ptr(np);
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  sweep_cl_config(h, nb, cfg, attr);
  int nc = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.dynamicSmemBytes) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc >= 1 ? nb : 0;
}

// Up to max_sweeps sweeps of the step in one cluster launch (grid from
// sweep_cl_grid); ends earlier when the step is done.
void launch_oci_sweep_cl(Handle &h, int grid, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps) {
  const int np = h.N / h.tune_P;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  sweep_cl_config(h, grid, cfg, attr);
#define OCI_SWEEP_CL(NP)                                                                                          \
  cudaLaunchKernelEx(&cfg, k_oci_sweep_cl<NP>, h.J, h.Jp, h.N, h.G, (const int32_t *)h.type,                     \
                     (const double *)h.tt.Linv, (const double *)h.tt.Mp, (const double *)h.inc,                 \
                     (const double *)h.tc, h.Psi[0], h.Psi[1], h.ds, h.e_hist, cond, use_cond,                  \
                     (const double *)h.tt.Win, (const double *)h.yc, (const double *)h.mu, max_sweeps)
  if (np == 2) OCI_SWEEP_CL(2);
  else if (np == 4) OCI_SWEEP_CL(4);
  else OCI_SWEEP_CL(8);
#undef OCI_SWEEP_CL
}

void launch_oci_sweep(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  // in the graph (or when the autotuner times it): all sweeps of the step in one launch where the blocks fit
  if (use_cond || h.mx_tune_sweeps > 0) {
    const int ncl = sweep_cl_grid(h);
    if (ncl > 0) {
      launch_oci_sweep_cl(h, ncl, cond, use_cond, h.mx_tune_sweeps > 0 ? h.mx_tune_sweeps : INT_MAX);
      return;
    }
    const int msg = sweep_ms_grid(h);
    if (msg > 0) {
      // in the graph: no sweep limit (the stop rule ends the step by max_iter at the latest)
      launch_oci_sweep_ms(h, msg, cond, use_cond, h.mx_tune_sweeps > 0 ? h.mx_tune_sweeps : INT_MAX);
      return;
    }
  }
  if (h.tune_reg && h.ordering != OCI_ORDER_RED_BLACK) {  // register form (Jacobi)
    const int cb = h.tune_cb, P = h.tune_P, np = h.N / P;
    const dim3 block(cb, h.G * P), grid((h.J + cb - 1) / cb);
    const size_t smem = sweep_reg_smem(h.G, cb, P);
#define OCI_SWEEP_REG(NP)                                                                                        \
  k_oci_sweep_reg<NP><<<grid, block, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Linv, h.tt.Cin, h.tt.Mp, \
                                                       h.w, h.inc, h.tc, h.Psi[0], h.Psi[1], h.ds, h.partials,   \
                                                       h.counter, h.e_hist, cond, use_cond, 0, (int)grid.x,      \
                                                       h.tt.Win, h.yc, h.mu)
    if (np == 2) OCI_SWEEP_REG(2);
    else if (np == 4) OCI_SWEEP_REG(4);
    else OCI_SWEEP_REG(8);
#undef OCI_SWEEP_REG
    return;
  }
  SweepCfg c = sweep_config(h);
  dim3 block(c.cells_per_block, h.G * c.chunks);
  if (h.ordering == OCI_ORDER_RED_BLACK && h.rb_pingpong && h.rb_cb > 0) {
    // the red-black shape timed at setup (staged or register form, ping-pong)
    const int cb = h.rb_cb, P = h.rb_P, half = (h.J + 1) / 2, grid = (half + cb - 1) / cb;
    const dim3 rblock(cb, h.G * P);
    if (!h.rb_reg) {
      const size_t smem = sweep_smem(h.N, h.G, cb, P, 8);
      for (int color = 0; color < 2; color++)
        k_oci_sweep_t<true, true><<<grid, rblock, smem, h.stream>>>(
            h.J, h.Jp, h.N, h.G, P, color, h.type, h.tt.Linv, h.tt.Cin, h.tt.Mp, h.w, h.inc, h.tc, h.Psi[0],
            h.Psi[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond, color == 1, 2 * grid);
      return;
    }
    const int np = h.N / P;
    const size_t smem = sweep_reg_smem(h.G, cb, P);
    for (int color = 0; color < 2; color++) {
#define OCI_SWEEP_REG_RB(NP)                                                                                     \
  k_oci_sweep_reg<NP, true><<<grid, rblock, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Linv, h.tt.Cin,   \
                                                              h.tt.Mp, h.w, h.inc, h.tc, h.Psi[0], h.Psi[1], h.ds, \
                                                              h.partials, h.counter, h.e_hist, cond, use_cond,     \
                                                              color, 2 * grid, h.tt.Win, h.yc, h.mu)
      if (np == 2) OCI_SWEEP_REG_RB(2);
      else if (np == 4) OCI_SWEEP_REG_RB(4);
      else OCI_SWEEP_REG_RB(8);
#undef OCI_SWEEP_REG_RB
    }
    return;
  }
  if (h.ordering == OCI_ORDER_RED_BLACK) {
    // two half sweeps, even cells then odd cells, each over ceil(J/2) threads;
    // the odd half reduces the partials of both
    const int half = (h.J + 1) / 2;
    const int grid = (half + c.cells_per_block - 1) / c.cells_per_block;
    for (int color = 0; color < 2; color++) {
      if (h.rb_pingpong)
        k_oci_sweep_t<true, true><<<grid, block, c.smem, h.stream>>>(
            h.J, h.Jp, h.N, h.G, c.chunks, color, h.type, h.tt.Linv, h.tt.Cin, h.tt.Mp, h.w, h.inc, h.tc, h.Psi[0],
            h.Psi[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond, color == 1, 2 * grid);
      else
        k_oci_sweep_t<true><<<grid, block, c.smem, h.stream>>>(
            h.J, h.Jp, h.N, h.G, c.chunks, color, h.type, h.tt.Linv, h.tt.Cin, h.tt.Mp, h.w, h.inc, h.tc, h.Psi[0],
            h.Psi[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond, color == 1, 2 * grid);
    }
    return;
  }
  k_oci_sweep_t<false><<<c.grid, block, c.smem, h.stream>>>(h.J, h.Jp, h.N, h.G, c.chunks, -1, h.type, h.tt.Linv,
                                                            h.tt.Cin, h.tt.Mp, h.w, h.inc, h.tc, h.Psi[0], h.Psi[1],
                                                            h.ds, h.partials, h.counter, h.e_hist, cond, use_cond, 1,
                                                            c.grid);
}

// One FP64 Jacobi sweep in two launches: part 0 the blocks that hold neither cell
// 0 nor cell J-1 (they read no incident flux), block partials only; part 1 the
// first and the last block, then the fixed-order sum of all block partials, the
// stop rule and the ping-pong flip.  Same cells, same partial slots and the same
// sum as one launch, so the same bits; between the parts the incident fluxes may
// change (a subdomain's halo arriving while its interior is swept).
void launch_oci_sweep_part(Handle &h, int part) {
  cudaGraphConditionalHandle none{};
  const bool reg = h.tune_reg != 0;
  const int cb = reg ? h.tune_cb : sweep_config(h).cells_per_block;
  const int nb = (h.J + cb - 1) / cb;
  int grid, boff, bstride, fuse;
  if (part == 0) {
    if (nb <= 2) return;  // no interior block
    grid = nb - 2, boff = 1, bstride = 1, fuse = 0;
  } else {
    grid = nb == 1 ? 1 : 2, boff = 0, bstride = nb == 1 ? 1 : nb - 1, fuse = 1;
  }
  if (reg) {
    const int P = h.tune_P, np = h.N / P;
    const dim3 block(cb, h.G * P);
    const size_t smem = sweep_reg_smem(h.G, cb, P);
#define OCI_SWEEP_REG_PART(NP)                                                                                     k_oci_sweep_reg<NP><<<grid, block, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Linv, h.tt.Cin, h.tt.Mp,                                                        h.w, h.inc, h.tc, h.Psi[0], h.Psi[1], h.ds, h.partials,                                                          h.counter, h.e_hist, none, 0, 0, nb, h.tt.Win, h.yc, h.mu,                                                         fuse, boff, bstride)
    if (np == 2) OCI_SWEEP_REG_PART(2);
    else if (np == 4) OCI_SWEEP_REG_PART(4);
    else OCI_SWEEP_REG_PART(8);
#undef OCI_SWEEP_REG_PART
    return;
  }
  SweepCfg c = sweep_config(h);
  dim3 block(c.cells_per_block, h.G * c.chunks);
  k_oci_sweep_t<false><<<grid, block, c.smem, h.stream>>>(h.J, h.Jp, h.N, h.G, c.chunks, -1, h.type, h.tt.Linv,
                                                          h.tt.Cin, h.tt.Mp, h.w, h.inc, h.tc, h.Psi[0], h.Psi[1],
                                                          h.ds, h.partials, h.counter, h.e_hist, none, 0, fuse, nb,
                                                          boff, bstride);
}

int sweep_partials(const Handle &h) {
  SweepCfg c = sweep_config(h);
  if (h.ordering == OCI_ORDER_RED_BLACK) {
    const int half = (h.J + 1) / 2;
    return 2 * ((half + c.cells_per_block - 1) / c.cells_per_block);
  }
  return c.grid;
}

// ------------------------------------------------------------------ a4, a5
// Sum the block partials in a fixed order, take e = sqrt(sum), apply the stop
// rule of Sec. 2.1 (Algorithm 2), flip the ping-pong index and, inside a
// conditional WHILE graph, end the loop when the step is done.
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const double *__restrict__ partials, int n,
                                                                 DevState *ds, double *e_hist,
                                                                 cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double red[32];
  if (ds->done) {
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double tot = block_sum_fixed(partials, n, red);
  if (threadIdx.x == 0) finish_fp64(ds, e_hist, sqrt(tot), cond, use_cond);
}

void launch_finalize(Handle &h, const double *partials, int n, cudaGraphConditionalHandle cond, int use_cond) {
  k_finalize<<<1, kFinalizeThreads, 0, h.stream>>>(partials, n, h.ds, h.e_hist, cond, use_cond);
}

// ------------------------------------------------------------------ a6
// Commit of a converged step: phi = sum_m w_m Psi (Eq. app:si_sf form),
// psi_{k-1/2} <- (Psi_hL, Psi_hR), and per-block particle-balance tallies:
//   time average (Eqs. scb-mb-a + b summed over corners, angles):
//     dx/(2 v dt) sum_{L,R}(phi_h - phi_prev) + leak + dx/2 St (phi_kL + phi_kR)
//       - dx/2 sum_gp Ss,gp->g (phi_gp,kL + phi_gp,kR) - dx/2 (Q_kL + Q_kR) = 0
//   time edge (Eqs. scb-mb-c + d):
//     dx/(v dt) sum_{L,R}(phi_h - phi_k) + leak + dx/2 St (phi_hL + phi_hR) - ... = 0
// partial layout [block][g][8] = {timeA, timeE, collA, collE, scatA, scatE, srcA, srcE}.
__global__ void __launch_bounds__(32 * kMaxG) k_carry(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                               const double *__restrict__ tdx, const double *__restrict__ tsig,
                                               const double *__restrict__ Kap, const double *__restrict__ v,
                                               double dt, const double *__restrict__ w,
                                               const double *__restrict__ Q, const double *Psi0,
                                               const double *Psi1, const DevState *__restrict__ ds,
                                               double *__restrict__ psi_prev, double *__restrict__ phi,
                                               double *__restrict__ bal_partials) {
  extern __shared__ double ph_sm[];  // [G*4][CB]
  const int CB = blockDim.x;
  const int cl = threadIdx.x, g = threadIdx.y;
  const int j = blockIdx.x * CB + cl;
  if (ds->status != OCI_OK) return;  // commit only a converged step (uniform)
  const bool active = j < J;
  const double *__restrict__ P = ds->cur ? Psi1 : Psi0;
  double ph[4] = {0, 0, 0, 0}, pp[2] = {0, 0};
  int tau = 0;
  if (active) {
    tau = type[j];
#pragma unroll 4
    for (int m = 0; m < N; m++) {
      const int gm = g * N + m;
      const double wm = w[m];
      const size_t base = (size_t)gm * 4 * Jp + j;
      double o[4];
#pragma unroll
      for (int p = 0; p < 4; p++) {
        o[p] = P[base + (size_t)p * Jp];
        ph[p] = fma(wm, o[p], ph[p]);
      }
      const size_t pb = (size_t)gm * 2 * Jp + j;
      pp[0] = fma(wm, psi_prev[pb], pp[0]);
      pp[1] = fma(wm, psi_prev[pb + Jp], pp[1]);
      psi_prev[pb] = o[2];
      psi_prev[pb + Jp] = o[3];
    }
#pragma unroll
    for (int p = 0; p < 4; p++) {
      phi[(size_t)(g * 4 + p) * Jp + j] = ph[p];
      ph_sm[(size_t)(g * 4 + p) * CB + cl] = ph[p];
    }
  }
  __syncthreads();
  double tally[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (active) {
    const double dx = tdx[tau];
    const double sig = tsig[(size_t)tau * G + g];
    const double rate = dx / (v[g] * dt);
    tally[0] = rate / 2.0 * ((ph[2] - pp[0]) + (ph[3] - pp[1]));
    tally[1] = rate * ((ph[2] - ph[0]) + (ph[3] - ph[1]));
    tally[2] = dx / 2.0 * sig * (ph[0] + ph[1]);
    tally[3] = dx / 2.0 * sig * (ph[2] + ph[3]);
    for (int gp = 0; gp < G; gp++) {
      const double k2 = 2.0 * Kap[((size_t)tau * G + gp) * G + g];  // dx/2 Sigma_s,gp->g
      tally[4] += k2 * (ph_sm[(size_t)(gp * 4 + 0) * CB + cl] + ph_sm[(size_t)(gp * 4 + 1) * CB + cl]);
      tally[5] += k2 * (ph_sm[(size_t)(gp * 4 + 2) * CB + cl] + ph_sm[(size_t)(gp * 4 + 3) * CB + cl]);
    }
    if (Q) {
      const double *q = Q + j;
      tally[6] = dx / 2.0 * (q[(size_t)(g * 4 + 0) * Jp] + q[(size_t)(g * 4 + 1) * Jp]);
      tally[7] = dx / 2.0 * (q[(size_t)(g * 4 + 2) * Jp] + q[(size_t)(g * 4 + 3) * Jp]);
    }
  }
  // reduce each tally over the 32 cells of each warp: one partial per 32 cells and group
  const size_t slot = (size_t)blockIdx.x * (CB / 32) + (cl >> 5);
#pragma unroll
  for (int k = 0; k < 8; k++) {
    double x = tally[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((cl & 31) == 0 && slot < (size_t)((J + 31) / 32))  // warps wholly past J own no slot
      bal_partials[(slot * G + g) * 8 + k] = x;
  }
}

// Sum the balance partials in a fixed order and add the leakage
// sum_m w_m mu_m (psi at x = X - psi at x = 0) with the upstream edge values.
constexpr int kBalThreads = 256;
__global__ void __launch_bounds__(kBalThreads) k_balance_final(int J, int Jp, int N, int G, int nblk, const double *__restrict__ bal_partials,
                                const double *__restrict__ mu, const double *__restrict__ w,
                                const double *__restrict__ inc, const double *Psi0, const double *Psi1,
                                const DevState *__restrict__ ds, double *__restrict__ bal) {
  const int g = blockIdx.x;
  constexpr int kT = kBalThreads;
  __shared__ double acc[8][kT];
  if (ds->status != OCI_OK) return;
  const int t = threadIdx.x;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = t; b < nblk; b += kT)
#pragma unroll
    for (int k = 0; k < 8; k++) s[k] += bal_partials[((size_t)b * G + g) * 8 + k];
  for (int k = 0; k < 8; k++) acc[k][t] = s[k];
  __syncthreads();
  for (int half = kT / 2; half > 0; half >>= 1) {  // fixed-order tree
    if (t < half)
      for (int k = 0; k < 8; k++) acc[k][t] += acc[k][t + half];
    __syncthreads();
  }
  if (t == 0) {
    double tot[8];
    for (int k = 0; k < 8; k++) tot[k] = acc[k][0];
    const double *P = ds->cur ? Psi1 : Psi0;
    double lA = 0.0, lE = 0.0;
    for (int m = 0; m < N; m++) {
      const int gm = g * N + m;
      double rk, rh, lk, lh;
      if (mu[m] > 0) {
        rk = P[(size_t)(gm * 4 + 1) * Jp + (J - 1)];
        rh = P[(size_t)(gm * 4 + 3) * Jp + (J - 1)];
        lk = inc[gm * 2 + 0];
        lh = inc[gm * 2 + 1];
      } else {
        lk = P[(size_t)(gm * 4 + 0) * Jp];
        lh = P[(size_t)(gm * 4 + 2) * Jp];
        rk = inc[(G * N + gm) * 2 + 0];
        rh = inc[(G * N + gm) * 2 + 1];
      }
      lA += w[m] * mu[m] * (rk - lk);
      lE += w[m] * mu[m] * (rh - lh);
    }
    double *bg = bal + (size_t)g * 10;
    bg[0] = tot[0]; bg[1] = lA; bg[2] = tot[2]; bg[3] = tot[4]; bg[4] = tot[6];
    bg[5] = tot[1]; bg[6] = lE; bg[7] = tot[3]; bg[8] = tot[5]; bg[9] = tot[7];
  }
}

void launch_carry(Handle &h) {
  // blocks of CB cells x G groups (at most 512 threads); balance partials per 32 cells
  int CB = 128;
  while (CB > 32 && CB * h.G > 512) CB /= 2;
  const int nblk = (h.J + 31) / 32;
  dim3 block(CB, h.G);
  k_carry<<<(h.J + CB - 1) / CB, block, (size_t)h.G * 4 * CB * sizeof(double), h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.dx, h.tt.sig, h.tt.Kap, h.v, h.dt, h.w,
                                        h.Q, h.Psi[0], h.Psi[1], h.ds, h.psi_prev, h.phi, h.bal_partials);
  k_balance_final<<<h.G, kBalThreads, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, nblk, h.bal_partials, h.mu, h.w, h.inc, h.Psi[0],
                                            h.Psi[1], h.ds, h.bal);
}

// ------------------------------------------------------------------ layout
// ABI [J][K] (K = G*N*P or G*4) <-> device [K][Jp], 32x32 tiles through shared memory.
__global__ void k_transpose_in(int J, int Jp, int K, const double *__restrict__ src, double *__restrict__ dst) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, k = k0 + threadIdx.x;
    tile[r][threadIdx.x] = (j < J && k < K) ? src[(size_t)j * K + k] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, j = j0 + threadIdx.x;
    if (k < K && j < Jp) dst[(size_t)k * Jp + j] = tile[threadIdx.x][r];
  }
}

__global__ void k_transpose_out(int J, int Jp, int K, const double *__restrict__ src, double *__restrict__ dst) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && j < J) ? src[(size_t)k * Jp + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, k = k0 + threadIdx.x;
    if (j < J && k < K) dst[(size_t)j * K + k] = tile[threadIdx.x][r];
  }
}

void launch_transpose_in(Handle &h, const double *src_abi, double *dst_soa, int K) {
  dim3 grid((K + 31) / 32, (h.Jp + 31) / 32);
  k_transpose_in<<<grid, dim3(32, 8), 0, h.stream>>>(h.J, h.Jp, K, src_abi, dst_soa);
}

void launch_transpose_out(Handle &h, const double *src_soa, double *dst_abi, int K) {
  dim3 grid((K + 31) / 32, (h.J + 31) / 32);
  k_transpose_out<<<grid, dim3(32, 8), 0, h.stream>>>(h.J, h.Jp, K, src_soa, dst_abi);
}

void launch_phi_out(Handle &h, double *dst_abi) { launch_transpose_out(h, h.phi, dst_abi, h.G * 4); }

// out[0:2K]  = (Psi_kL, Psi_hL) of cell 0 per (g,m);
// out[2K:4K] = (Psi_kR, Psi_hR) of cell J-1 per (g,m); K = G*N.
__global__ void k_edges(int J, int Jp, int K, const double *__restrict__ P, double *__restrict__ out) {
  const int gm = blockIdx.x * blockDim.x + threadIdx.x;
  if (gm >= K) return;
  const size_t b = (size_t)gm * 4 * Jp;
  out[gm * 2 + 0] = P[b + 0 * (size_t)Jp];
  out[gm * 2 + 1] = P[b + 2 * (size_t)Jp];
  out[2 * K + gm * 2 + 0] = P[b + 1 * (size_t)Jp + (J - 1)];
  out[2 * K + gm * 2 + 1] = P[b + 3 * (size_t)Jp + (J - 1)];
}

void launch_edges(Handle &h, const double *Psi, double *out) {
  const int K = h.G * h.N;
  k_edges<<<(K + 127) / 128, 128, 0, h.stream>>>(h.J, h.Jp, K, Psi, out);
}

}  // namespace oci
