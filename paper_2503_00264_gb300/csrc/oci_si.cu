// oci_si.cu -- source iteration (SI) comparison path, FP64 (Algorithm 1, App. A).
//
// One SI sweep solves, for every (g,m) and cell j in the direction of flight,
//   L_{c,j,g,m} psi_j = d_j,   d_j = d0_j + |mu| (u_k e_a + u_h e_b)      (Eq. app:si_sys)
// with d0 = dx/4 (sum_gp Sigma_s,gp->g phi^(l)_gp + Q) + dx/(2 v dt) (psi_prev_L, psi_prev_R, 0, 0)
// (Eq. app:si_rhs; all groups' scattering lagged = Jacobi over groups) and the
// upstream edge (u_k, u_h) of the CURRENT sweep (rows a,b = 0,2 for mu > 0 and
// 1,3 for mu < 0).  Writing z_j = L^{-1} d0_j, the solution is
//   psi_j = z_j + Cin_j u_j
// so the serial dependency of the sweep is only the two outgoing edge values,
//   u_{next} = z_j[out] + Cin_j[out,:] u_j       (2 dependent FMA levels per cell).
// The sweep is split into a parallel pre-pass (z), a serial chain per (g,m)
// (one block each, one walking thread fed from shared memory), and a parallel
// post-pass (psi, phi, ||phi^{l+1}-phi^l||^2).
#include <math.h>

#include "oci_internal.h"

namespace oci {

// Scattering + fixed source of every (j,g): src_p = dx/4 (sum_gp Ss,gp->g phi_gp,p + Q_g,p),
// folded with the time term into d0 and pre-multiplied by L^{-1}: z = L^{-1} d0.
__global__ void k_si_pre(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                         const double *__restrict__ tdx, const double *__restrict__ Kap,
                         const double *__restrict__ v, double dt, const double *__restrict__ Q,
                         const double *__restrict__ psi_prev, const double *__restrict__ Linv,
                         const double *phi0, const double *phi1, const DevState *__restrict__ ds,
                         double *__restrict__ z) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (j >= J || ds->done) return;
  const double *__restrict__ phl = ds->cur ? phi1 : phi0;
  const int tau = type[j];
  const double dx = tdx[tau];
  double s[4];
#pragma unroll
  for (int p = 0; p < 4; p++) s[p] = Q ? dx / 4.0 * Q[(size_t)(g * 4 + p) * Jp + j] : 0.0;
  for (int gp = 0; gp < G; gp++) {
    const double k = Kap[((size_t)tau * G + gp) * G + g];
#pragma unroll
    for (int p = 0; p < 4; p++) s[p] = fma(k, phl[(size_t)(gp * 4 + p) * Jp + j], s[p]);
  }
  const double ah = dx / (2.0 * v[g] * dt);
  for (int m = 0; m < N; m++) {
    const int gm = g * N + m;
    const double d0 = s[0] + ah * psi_prev[(size_t)(gm * 2 + 0) * Jp + j];
    const double d1 = s[1] + ah * psi_prev[(size_t)(gm * 2 + 1) * Jp + j];
    const double *L = Linv + ((size_t)tau * G * N + gm) * 16;
#pragma unroll
    for (int p = 0; p < 4; p++)
      z[(size_t)(gm * 4 + p) * Jp + j] = L[p * 4 + 0] * d0 + L[p * 4 + 1] * d1 + L[p * 4 + 2] * s[2] + L[p * 4 + 3] * s[3];
  }
}

// Serial chain of one (g,m), one block per chain: the block's threads stage the
// next chunk of cells (the two outgoing rows of z and of Cin, in sweep order)
// into shared memory while thread 0 walks the current chunk, so the walk sees
// only shared-memory loads and its 2 dependent FMA levels per cell.  The
// incoming edge of every cell is buffered and written back by all threads.
constexpr int kChainChunk = 256;
constexpr int kChainThreads = 128;
__global__ void __launch_bounds__(kChainThreads) k_si_chain(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                                            const double *__restrict__ Cin,
                                                            const double *__restrict__ inc,
                                                            const double *__restrict__ z,
                                                            const DevState *__restrict__ ds,
                                                            double *__restrict__ uin) {
  __shared__ double sa[2][kChainChunk], sb[2][kChainChunk], sc[2][4][kChainChunk];
  __shared__ double su[2][kChainChunk];
  const int gm = blockIdx.x;
  if (gm >= G * N || ds->done) return;
  const int m = gm % N;
  const bool fwd = m >= N / 2;  // mu > 0: sweep j = 0 .. J-1
  const int oa = fwd ? 1 : 0;   // outgoing rows: R corners (mu > 0) or L corners (mu < 0)
  const int ob = fwd ? 3 : 2;
  const double *za = z + (size_t)(gm * 4 + oa) * Jp;
  const double *zb = z + (size_t)(gm * 4 + ob) * Jp;
  double *uk_out = uin + (size_t)(gm * 2 + 0) * Jp;
  double *uh_out = uin + (size_t)(gm * 2 + 1) * Jp;
  const int nchunk = (J + kChainChunk - 1) / kChainChunk;
  auto stage = [&](int ck, int buf) {
    for (int i = threadIdx.x; i < kChainChunk; i += kChainThreads) {
      const int s = ck * kChainChunk + i;
      if (s < J) {
        const int j = fwd ? s : J - 1 - s;
        sa[buf][i] = za[j];
        sb[buf][i] = zb[j];
        const double *C = Cin + ((size_t)type[j] * G * N + gm) * 8;
        sc[buf][0][i] = C[oa * 2 + 0];
        sc[buf][1][i] = C[oa * 2 + 1];
        sc[buf][2][i] = C[ob * 2 + 0];
        sc[buf][3][i] = C[ob * 2 + 1];
      }
    }
  };
  auto flush = [&](int ck, int buf) {  // write back the incoming edges of chunk ck
    for (int i = threadIdx.x; i < kChainChunk; i += kChainThreads) {
      const int s = ck * kChainChunk + i;
      if (s < J) {
        const int j = fwd ? s : J - 1 - s;
        uk_out[j] = su[buf][i];
      }
    }
  };
  const double *incp = inc + (fwd ? 0 : (size_t)G * N * 2) + gm * 2;
  double uk = incp[0], uh = incp[1];
  stage(0, 0);
  __syncthreads();
  __shared__ double suh[2][kChainChunk];
  for (int ck = 0; ck < nchunk; ck++) {
    const int buf = ck & 1;
    if (ck + 1 < nchunk) stage(ck + 1, buf ^ 1);
    if (threadIdx.x == 0) {
      const int cnt = min(kChainChunk, J - ck * kChainChunk);
      for (int i = 0; i < cnt; i++) {
        su[buf][i] = uk;
        suh[buf][i] = uh;
        const double nk = fma(sc[buf][1][i], uh, fma(sc[buf][0][i], uk, sa[buf][i]));
        const double nh = fma(sc[buf][3][i], uh, fma(sc[buf][2][i], uk, sb[buf][i]));
        uk = nk;
        uh = nh;
      }
    }
    __syncthreads();
    flush(ck, buf);
    for (int i = threadIdx.x; i < kChainChunk; i += kChainThreads) {
      const int s = ck * kChainChunk + i;
      if (s < J) uh_out[fwd ? s : J - 1 - s] = suh[buf][i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- scan form
// The chain of one (g,m) is a composition of affine maps of the outgoing edge,
//   u_{s+1} = F_s(u_s) = B_s u_s + a_s,   B_s = Cin_j[out rows], a_s = z_j[out rows],
// and affine maps compose associatively: (F2 o F1)(u) = B2 B1 u + (B2 a1 + a2).
// The scan form computes the same incoming edges in three parallel passes:
//   1. every segment of kScanSeg cells (one thread per (g,m), segment) composes
//      its maps into one affine map;
//   2. one thread per (g,m) applies the segment maps in order to get each
//      segment's incoming edge;
//   3. every segment walks its cells again from its incoming edge.
// The result equals the sequential sweep up to rounding (a different
// association of the same products).
constexpr int kScanSeg = 128;

__device__ __forceinline__ void si_cell_map(int j, int gm, int G, int N, int oa, int ob,
                                            const int32_t *__restrict__ type, const double *__restrict__ Cin,
                                            const double *__restrict__ za, const double *__restrict__ zb,
                                            double B[4], double a[2]) {
  const double *C = Cin + ((size_t)type[j] * G * N + gm) * 8;
  B[0] = C[oa * 2 + 0];
  B[1] = C[oa * 2 + 1];
  B[2] = C[ob * 2 + 0];
  B[3] = C[ob * 2 + 1];
  a[0] = za[j];
  a[1] = zb[j];
}

__global__ void k_si_seg_maps(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                              const double *__restrict__ Cin, const double *__restrict__ z,
                              const DevState *__restrict__ ds, double *__restrict__ maps) {
  const int K = (J + kScanSeg - 1) / kScanSeg;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= G * N * K || ds->done) return;
  const int gm = tid / K, seg = tid % K;
  const int m = gm % N;
  const bool fwd = m >= N / 2;
  const int oa = fwd ? 1 : 0, ob = fwd ? 3 : 2;
  const double *za = z + (size_t)(gm * 4 + oa) * Jp;
  const double *zb = z + (size_t)(gm * 4 + ob) * Jp;
  double M0 = 1.0, M1 = 0.0, M2 = 0.0, M3 = 1.0, m0 = 0.0, m1 = 0.0;  // identity map
  const int s1 = min(J, (seg + 1) * kScanSeg);
  for (int s = seg * kScanSeg; s < s1; s++) {
    const int j = fwd ? s : J - 1 - s;
    double B[4], a[2];
    si_cell_map(j, gm, G, N, oa, ob, type, Cin, za, zb, B, a);
    // M <- F_s o M
    const double n0 = fma(B[0], M0, B[1] * M2), n1 = fma(B[0], M1, B[1] * M3);
    const double n2 = fma(B[2], M0, B[3] * M2), n3 = fma(B[2], M1, B[3] * M3);
    const double v0 = fma(B[0], m0, fma(B[1], m1, a[0]));
    const double v1 = fma(B[2], m0, fma(B[3], m1, a[1]));
    M0 = n0; M1 = n1; M2 = n2; M3 = n3; m0 = v0; m1 = v1;
  }
  double *o = maps + (size_t)tid * 6;
  o[0] = M0; o[1] = M1; o[2] = M2; o[3] = M3; o[4] = m0; o[5] = m1;
}

__global__ void k_si_seg_scan(int J, int N, int G, const double *__restrict__ inc, const double *__restrict__ maps,
                              const DevState *__restrict__ ds, double *__restrict__ segin) {
  const int K = (J + kScanSeg - 1) / kScanSeg;
  const int gm = blockIdx.x * blockDim.x + threadIdx.x;
  if (gm >= G * N || ds->done) return;
  const int m = gm % N;
  const bool fwd = m >= N / 2;
  const double *incp = inc + (fwd ? 0 : (size_t)G * N * 2) + gm * 2;
  double uk = incp[0], uh = incp[1];
  for (int seg = 0; seg < K; seg++) {
    const double *M = maps + ((size_t)gm * K + seg) * 6;
    segin[((size_t)gm * K + seg) * 2 + 0] = uk;
    segin[((size_t)gm * K + seg) * 2 + 1] = uh;
    const double nk = fma(M[0], uk, fma(M[1], uh, M[4]));
    const double nh = fma(M[2], uk, fma(M[3], uh, M[5]));
    uk = nk;
    uh = nh;
  }
}

__global__ void k_si_seg_walk(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                              const double *__restrict__ Cin, const double *__restrict__ z,
                              const double *__restrict__ segin, const DevState *__restrict__ ds,
                              double *__restrict__ uin) {
  const int K = (J + kScanSeg - 1) / kScanSeg;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= G * N * K || ds->done) return;
  const int gm = tid / K, seg = tid % K;
  const int m = gm % N;
  const bool fwd = m >= N / 2;
  const int oa = fwd ? 1 : 0, ob = fwd ? 3 : 2;
  const double *za = z + (size_t)(gm * 4 + oa) * Jp;
  const double *zb = z + (size_t)(gm * 4 + ob) * Jp;
  double *uk_out = uin + (size_t)(gm * 2 + 0) * Jp;
  double *uh_out = uin + (size_t)(gm * 2 + 1) * Jp;
  double uk = segin[(size_t)tid * 2 + 0], uh = segin[(size_t)tid * 2 + 1];
  const int s1 = min(J, (seg + 1) * kScanSeg);
  for (int s = seg * kScanSeg; s < s1; s++) {
    const int j = fwd ? s : J - 1 - s;
    double B[4], a[2];
    si_cell_map(j, gm, G, N, oa, ob, type, Cin, za, zb, B, a);
    uk_out[j] = uk;
    uh_out[j] = uh;
    const double nk = fma(B[1], uh, fma(B[0], uk, a[0]));
    const double nh = fma(B[3], uh, fma(B[2], uk, a[1]));
    uk = nk;
    uh = nh;
  }
}

size_t si_scan_maps(const Handle &h) {
  const size_t K = (h.J + kScanSeg - 1) / kScanSeg;
  return (size_t)h.G * h.N * K;
}

// psi_j = z_j + Cin_j u_j for all (g,m); phi^{l+1}; block sum of (phi^{l+1} - phi^l)^2.
__global__ void __launch_bounds__(256) k_si_post(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                                 const double *__restrict__ Cin, const double *__restrict__ w,
                                                 const double *__restrict__ z, const double *__restrict__ uin,
                                                 double *Psi0, double *Psi1, double *phi0, double *phi1,
                                                 const DevState *__restrict__ ds, double *__restrict__ partials) {
  __shared__ double red[32];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (ds->done) return;
  const int cur = ds->cur;
  double *__restrict__ Pout = cur ? Psi0 : Psi1;
  const double *__restrict__ phl = cur ? phi1 : phi0;
  double *__restrict__ phn = cur ? phi0 : phi1;
  double e2 = 0.0;
  if (j < J) {
    const int tau = type[j];
    double ph[4] = {0, 0, 0, 0};
    for (int m = 0; m < N; m++) {
      const int gm = g * N + m;
      const double uk = uin[(size_t)(gm * 2 + 0) * Jp + j];
      const double uh = uin[(size_t)(gm * 2 + 1) * Jp + j];
      const double *C = Cin + ((size_t)tau * G * N + gm) * 8;
      const double wm = w[m];
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const size_t ix = (size_t)(gm * 4 + p) * Jp + j;
        const double o = fma(C[p * 2 + 1], uh, fma(C[p * 2 + 0], uk, z[ix]));
        Pout[ix] = o;
        ph[p] = fma(wm, o, ph[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < 4; p++) {
      const size_t ix = (size_t)(g * 4 + p) * Jp + j;
      const double d = ph[p] - phl[ix];
      e2 = fma(d, d, e2);
      phn[ix] = ph[p];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; i++) s += red[i];
    partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// phi[cur] = sum_m w_m Psi[cur] (initial SI iterate from the handle's Psi).
__global__ void k_si_phi_init(int J, int Jp, int N, int G, const double *__restrict__ w, const double *Psi0,
                              const double *Psi1, double *phi0, double *phi1, const DevState *__restrict__ ds) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (j >= J) return;
  const int cur = ds->cur;
  const double *P = cur ? Psi1 : Psi0;
  double *ph = cur ? phi1 : phi0;
  double s[4] = {0, 0, 0, 0};
  for (int m = 0; m < N; m++) {
#pragma unroll
    for (int p = 0; p < 4; p++) s[p] = fma(w[m], P[(size_t)((g * N + m) * 4 + p) * Jp + j], s[p]);
  }
#pragma unroll
  for (int p = 0; p < 4; p++) ph[(size_t)(g * 4 + p) * Jp + j] = s[p];
}

void launch_si_sweep(Handle &h) {
  dim3 g1((h.J + 255) / 256, h.G);
  k_si_pre<<<g1, 256, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.dx, h.tt.Kap, h.v, h.dt, h.Q, h.psi_prev,
                                     h.tt.Linv, h.phi_si[0], h.phi_si[1], h.ds, h.si_z);
  if (h.si_mode == OCI_SI_SCAN) {
    const int nmaps = (int)si_scan_maps(h);
    k_si_seg_maps<<<(nmaps + 127) / 128, 128, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Cin, h.si_z, h.ds,
                                                             h.si_maps);
    k_si_seg_scan<<<(h.G * h.N + 31) / 32, 32, 0, h.stream>>>(h.J, h.N, h.G, h.inc, h.si_maps, h.ds, h.si_segin);
    k_si_seg_walk<<<(nmaps + 127) / 128, 128, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Cin, h.si_z,
                                                             h.si_segin, h.ds, h.si_uin);
  } else {
    k_si_chain<<<h.G * h.N, kChainThreads, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Cin, h.inc, h.si_z,
                                                            h.ds, h.si_uin);
  }
  k_si_post<<<g1, 256, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Cin, h.w, h.si_z, h.si_uin, h.Psi[0],
                                      h.Psi[1], h.phi_si[0], h.phi_si[1], h.ds, h.partials);
}

int si_partials(const Handle &h) { return ((h.J + 255) / 256) * h.G; }

void launch_si_phi_from_psi(Handle &h, double *) {
  dim3 g1((h.J + 255) / 256, h.G);
  k_si_phi_init<<<g1, 256, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.w, h.Psi[0], h.Psi[1], h.phi_si[0], h.phi_si[1],
                                          h.ds);
}

}  // namespace oci
