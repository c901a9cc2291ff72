// oci_dense.cu -- per-cell dense path (factor once, solve every sweep), FP64.
//
// This is the paper's scheme (Algorithm 2: gesv on the first iteration, getrs
// afterwards) rebuilt for one GPU: every cell's dense A_j of order n = 4NG
// (Eqs. Aja, Aj, scatter_mg, fullOCIlhs) is assembled on the device, factored
// once by a warp-cooperative LU with partial pivoting, and every sweep applies
// one forward and one back substitution per cell (one warp per cell).  It needs
// no cell sharing, so it serves slabs whose cells all differ.
//
// Storage: LU[j] column-major (element (r,c) at c*n + r) so that a warp's lanes
// read consecutive rows of one column; perm[j][i] = row of b that lands in
// position i after the pivoting row swaps.
//
// Default apply: the inverse.  The triangular solves of getrs move one column
// at a time and each column depends on the previous one, so on this part --
// whose FP64 pipe retires 2 FMA per SM and clock -- a warp-per-cell
// substitution leaves a third of the lanes idle (columns shorter than 32 rows)
// and waits on a global load per column.  The same factor-once / apply-every-
// sweep scheme with the explicit inverse A_j^{-1}, formed once at setup by
// Gauss-Jordan elimination with partial pivoting (k_dense_invert, the cell's
// matrix staged in shared memory), costs the same 2 n^2 flops and 8 n^2 bytes
// per cell and sweep as the two triangular solves, but is a plain matrix-vector
// product (k_dense_apply): every lane owns rows, the column loads do not depend
// on earlier results and can all be in flight.  OCI_DENSE_APPLY=lu (a test
// hook) keeps the LU factors and the triangular solves instead.
#include <math.h>

#include "oci_internal.h"

namespace oci {

// A_j, column-major.  Row/column index u = (g*N+m)*4+p.
__global__ void k_dense_assemble(int J, int N, int G, const int32_t *__restrict__ type,
                                 const double *__restrict__ tdx, const double *__restrict__ tsig,
                                 const double *__restrict__ Kap, const double *__restrict__ v, double dt,
                                 const double *__restrict__ mu, const double *__restrict__ w,
                                 double *__restrict__ LU) {
  const int j = blockIdx.x;
  const int n = 4 * N * G;
  const int tau = type[j];
  const double dx = tdx[tau];
  double *A = LU + (size_t)j * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int c = e / n, r = e % n;
    const int gr = r / (4 * N), mr = (r / 4) % N, pr = r % 4;
    const int gc = c / (4 * N), mc = (c / 4) % N, pc = c % 4;
    double a = 0.0;
    if (gr == gc && mr == mc) {
      const double m_ = mu[mr];
      const double al = dx / (v[gr] * dt);
      const double d = (fabs(m_) + dx * tsig[(size_t)tau * G + gr]) / 2.0;
      // L_{c,j,g,m} of Eq. Aj
      const double L[16] = {d,      m_ / 2.0, al / 2.0,  0.0,      -m_ / 2.0, d,        0.0,      al / 2.0,
                            -al,    0.0,      al + d,    m_ / 2.0, 0.0,       -al,      -m_ / 2.0, al + d};
      a = L[pr * 4 + pc];
    }
    if (pr == pc) a -= Kap[((size_t)tau * G + gc) * G + gr] * w[mc];  // dx/4 Sigma_s,gc->gr w_mc
    A[e] = a;
  }
}

// Warp-cooperative LU with partial pivoting (first largest |pivot| on ties),
// in place; one warp per cell.  Sets *singular if a pivot column is zero.
__global__ void k_dense_factor(int J, int n, double *__restrict__ LU, int32_t *__restrict__ perm,
                               int *__restrict__ singular) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= J) return;
  double *A = LU + (size_t)j * n * n;
  int32_t *P = perm + (size_t)j * n;
  for (int i = lane; i < n; i += 32) P[i] = i;
  __syncwarp();
  for (int k = 0; k < n; k++) {
    double best = -1.0;
    int br = k;
    for (int i = k + lane; i < n; i += 32) {
      const double a = fabs(A[(size_t)k * n + i]);
      if (a > best) {
        best = a;
        br = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int orow = __shfl_xor_sync(0xffffffffu, br, o);
      if (ob > best || (ob == best && orow < br)) {
        best = ob;
        br = orow;
      }
    }
    if (best == 0.0) {
      if (lane == 0) atomicExch(singular, 1);
      return;
    }
    if (br != k) {
      for (int c = lane; c < n; c += 32) {
        const double t = A[(size_t)c * n + k];
        A[(size_t)c * n + k] = A[(size_t)c * n + br];
        A[(size_t)c * n + br] = t;
      }
      if (lane == 0) {
        const int t = P[k];
        P[k] = P[br];
        P[br] = t;
      }
    }
    __syncwarp();
    const double piv = A[(size_t)k * n + k];
    for (int i = k + 1 + lane; i < n; i += 32) A[(size_t)k * n + i] /= piv;
    __syncwarp();
    for (int c = k + 1; c < n; c++) {
      const double akc = A[(size_t)c * n + k];
      for (int i = k + 1 + lane; i < n; i += 32) A[(size_t)c * n + i] -= A[(size_t)k * n + i] * akc;
    }
    __syncwarp();
  }
}

// In-place Gauss-Jordan inversion with partial pivoting (first largest |pivot|),
// one warp per cell, the column-major cell matrix staged in shared memory.
// Step k: swap rows k and p (the pivot row), scale row k by 1/a_kk (storing
// 1/a_kk at (k,k)), eliminate column k from every other row (storing
// -a_rk/a_kk at (r,k)); afterwards the columns are swapped back in reverse
// order of the row swaps.  Sets *singular if a pivot is zero or not finite.
__global__ void __launch_bounds__(64) k_dense_invert(int J, int n, double *__restrict__ Ainv,
                                                     int *__restrict__ singular) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int j = blockIdx.x * nw + wid;
  double *A = sm + (size_t)wid * ((size_t)n * n + n);  // [n][n] column-major, then f[n]
  double *f = A + (size_t)n * n;
  int *sw = (int *)(sm + (size_t)nw * ((size_t)n * n + n)) + (size_t)wid * n;
  if (j >= J) return;  // whole warp: no block-wide barrier below
  double *G = Ainv + (size_t)j * n * n;
  for (int e = lane; e < n * n; e += 32) A[e] = G[e];
  __syncwarp();
  bool bad = false;
  for (int k = 0; k < n && !bad; k++) {
    double best = -1.0;
    int br = k;
    for (int i = k + lane; i < n; i += 32) {
      const double a = fabs(A[(size_t)k * n + i]);
      if (a > best) {
        best = a;
        br = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int orow = __shfl_xor_sync(0xffffffffu, br, o);
      if (ob > best || (ob == best && orow < br)) {
        best = ob;
        br = orow;
      }
    }
    if (!(best > 0.0) || !isfinite(best)) {
      bad = true;
      break;
    }
    if (lane == 0) sw[k] = br;
    if (br != k)
      for (int c = lane; c < n; c += 32) {
        const double t = A[(size_t)c * n + k];
        A[(size_t)c * n + k] = A[(size_t)c * n + br];
        A[(size_t)c * n + br] = t;
      }
    __syncwarp();
    const double inv = 1.0 / A[(size_t)k * n + k];
    for (int r = lane; r < n; r += 32) f[r] = A[(size_t)k * n + r];  // column k before elimination
    __syncwarp();
    for (int c = lane; c < n; c += 32) A[(size_t)c * n + k] = c == k ? inv : A[(size_t)c * n + k] * inv;  // row k
    __syncwarp();
    for (int c = 0; c < n; c++) {
      const double akc = A[(size_t)c * n + k];
      for (int r = lane; r < n; r += 32) {
        if (r == k) continue;
        A[(size_t)c * n + r] = c == k ? -f[r] * inv : fma(-f[r], akc, A[(size_t)c * n + r]);
      }
    }
    __syncwarp();
  }
  if (bad) {
    if (lane == 0) atomicExch(singular, 1);
    return;
  }
  for (int k = n - 1; k >= 0; k--) {  // undo the row swaps on the columns
    const int p = sw[k];
    if (p != k)
      for (int r = lane; r < n; r += 32) {
        const double t = A[(size_t)k * n + r];
        A[(size_t)k * n + r] = A[(size_t)p * n + r];
        A[(size_t)p * n + r] = t;
      }
    __syncwarp();
  }
  for (int e = lane; e < n * n; e += 32) G[e] = A[e];
}

// Shared memory of k_dense_invert with nw warps (cells) per block.
size_t dense_invert_smem(int n, int nw) { return (size_t)nw * ((size_t)n * n + n) * 8 + (size_t)nw * n * 4; }

// Per-step constant c = [dx/4 Q_kL + dx/(2v dt) psi_prev_L, dx/4 Q_kR + ..., dx/4 Q_hL, dx/4 Q_hR].
__global__ void k_dense_step_const(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                   const double *__restrict__ tdx, const double *__restrict__ v, double dt,
                                   const double *__restrict__ Q, const double *__restrict__ psi_prev,
                                   double *__restrict__ cvec) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int gm = blockIdx.y;
  if (j >= J) return;
  const int g = gm / N;
  const double dx = tdx[type[j]];
  const double ah = dx / (2.0 * v[g] * dt);
#pragma unroll
  for (int p = 0; p < 4; p++) {
    double c = Q ? dx / 4.0 * Q[(size_t)(g * 4 + p) * Jp + j] : 0.0;
    if (p < 2) c += ah * psi_prev[(size_t)(gm * 2 + p) * Jp + j];
    cvec[(size_t)(gm * 4 + p) * Jp + j] = c;
  }
}

// One sweep: b_j = c_j + lagged inflow (Eq. rhs_sg), Psi_j = U^{-1} L^{-1} P b_j.
constexpr int kDenseWarps = 8;
constexpr int kDenseMaxNQ = 8;  // inverse apply: rows per lane, so n <= 256
__global__ void __launch_bounds__(kDenseWarps * 32) k_dense_sweep(
    int J, int Jp, int N, int G, const double *__restrict__ LU, const int32_t *__restrict__ perm,
    const double *__restrict__ mu, const double *__restrict__ inc, const double *__restrict__ cvec,
    double *Psi0, double *Psi1, const DevState *__restrict__ ds, double *__restrict__ partials) {
  extern __shared__ double sm[];
  __shared__ double red[kDenseWarps];
  const int n = 4 * N * G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.x * kDenseWarps + wid;
  if (ds->done) return;
  const int cur = ds->cur;
  const double *__restrict__ Pin = cur ? Psi1 : Psi0;
  double *__restrict__ Pout = cur ? Psi0 : Psi1;
  double *b = sm + (size_t)wid * 2 * n;
  double *x = b + n;
  double e2 = 0.0;
  if (j < J) {
    for (int u = lane; u < n; u += 32) {
      const int gm = u >> 2, p = u & 3, m = gm % N;
      double val = cvec[(size_t)u * Jp + j];
      if (mu[m] > 0) {
        if (p == 0 || p == 2) {
          const double up = j > 0 ? Pin[(size_t)(gm * 4 + p + 1) * Jp + j - 1] : inc[gm * 2 + (p >> 1)];
          val = fma(mu[m], up, val);
        }
      } else {
        if (p == 1 || p == 3) {
          const double up = j < J - 1 ? Pin[(size_t)(gm * 4 + p - 1) * Jp + j + 1] : inc[(G * N + gm) * 2 + (p >> 1)];
          val = fma(-mu[m], up, val);
        }
      }
      b[u] = val;
    }
    __syncwarp();
    const double *A = LU + (size_t)j * n * n;
    const int32_t *P = perm + (size_t)j * n;
    for (int i = lane; i < n; i += 32) x[i] = b[P[i]];
    __syncwarp();
    // forward substitution with the unit lower factor
    for (int k = 0; k < n - 1; k++) {
      const double xk = x[k];
      const double *col = A + (size_t)k * n;
      for (int i = k + 1 + lane; i < n; i += 32) x[i] = fma(-col[i], xk, x[i]);
      __syncwarp();
    }
    // back substitution with the upper factor
    for (int k = n - 1; k >= 0; k--) {
      const double *col = A + (size_t)k * n;
      const double xk = x[k] / col[k];
      __syncwarp();
      if (lane == (k & 31)) x[k] = xk;
      for (int i = lane; i < k; i += 32) x[i] = fma(-col[i], xk, x[i]);
      __syncwarp();
    }
    for (int u = lane; u < n; u += 32) {
      const size_t ix = (size_t)u * Jp + j;
      const double d = x[u] - Pin[ix];
      e2 = fma(d, d, e2);
      Pout[ix] = x[u];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
  if (lane == 0) red[wid] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kDenseWarps; i++) s += red[i];
    partials[blockIdx.x] = s;
  }
}

// One sweep with the explicit inverse: b_j as in k_dense_sweep, Psi_j = A_j^{-1} b_j
// as a matrix-vector product, one warp per cell, lane l owning rows l, l+32, ...
// (NQ rows at most); the columns of A_j^{-1} are read in order, eight at a time.
template <int NQ>
__global__ void __launch_bounds__(kDenseWarps * 32) k_dense_apply(
    int J, int Jp, int N, int G, const double *__restrict__ Ainv, const double *__restrict__ mu,
    const double *__restrict__ inc, const double *__restrict__ cvec, double *Psi0, double *Psi1,
    const DevState *__restrict__ ds, double *__restrict__ partials) {
  extern __shared__ double sm[];
  __shared__ double red[kDenseWarps];
  const int n = 4 * N * G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.x * kDenseWarps + wid;
  if (ds->done) return;
  const int cur = ds->cur;
  const double *__restrict__ Pin = cur ? Psi1 : Psi0;
  double *__restrict__ Pout = cur ? Psi0 : Psi1;
  double *b = sm + (size_t)wid * n;
  double e2 = 0.0;
  if (j < J) {
    for (int u = lane; u < n; u += 32) {
      const int gm = u >> 2, p = u & 3, m = gm % N;
      double val = cvec[(size_t)u * Jp + j];
      if (mu[m] > 0) {
        if (p == 0 || p == 2) {
          const double up = j > 0 ? Pin[(size_t)(gm * 4 + p + 1) * Jp + j - 1] : inc[gm * 2 + (p >> 1)];
          val = fma(mu[m], up, val);
        }
      } else {
        if (p == 1 || p == 3) {
          const double up = j < J - 1 ? Pin[(size_t)(gm * 4 + p - 1) * Jp + j + 1] : inc[(G * N + gm) * 2 + (p >> 1)];
          val = fma(-mu[m], up, val);
        }
      }
      b[u] = val;
    }
    __syncwarp();
    const double *__restrict__ A = Ainv + (size_t)j * n * n;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] = 0.0;
    int k = 0;
    for (; k + 8 <= n; k += 8) {
      double a[8][NQ];
#pragma unroll
      for (int t = 0; t < 8; t++)
#pragma unroll
        for (int q = 0; q < NQ; q++) {
          const int r = lane + 32 * q;
          a[t][q] = r < n ? A[(size_t)(k + t) * n + r] : 0.0;
        }
#pragma unroll
      for (int t = 0; t < 8; t++) {
        const double bk = b[k + t];
#pragma unroll
        for (int q = 0; q < NQ; q++) acc[q] = fma(a[t][q], bk, acc[q]);
      }
    }
    for (; k < n; k++) {
      const double bk = b[k];
#pragma unroll
      for (int q = 0; q < NQ; q++) {
        const int r = lane + 32 * q;
        if (r < n) acc[q] = fma(A[(size_t)k * n + r], bk, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) {
      const int u = lane + 32 * q;
      if (u < n) {
        const size_t ix = (size_t)u * Jp + j;
        const double d = acc[q] - Pin[ix];
        e2 = fma(d, d, e2);
        Pout[ix] = acc[q];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
  if (lane == 0) red[wid] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kDenseWarps; i++) s += red[i];
    partials[blockIdx.x] = s;
  }
}

int dense_setup(Handle &h) {
  const int n = 4 * h.N * h.G;
  const size_t bytes = (size_t)h.J * n * n * sizeof(double);
  const size_t smem = (size_t)kDenseWarps * 2 * n * sizeof(double);
  const char *ap = hook_env("OCI_DENSE_APPLY");
  const int inv_w = dense_invert_smem(n, 2) <= 200 * 1024 ? 2 : 1;  // cells per inversion block
  h.dense_inv = !(ap && ap[0] == 'l') && n <= 32 * kDenseMaxNQ && dense_invert_smem(n, 1) <= 200 * 1024;
  cudaError_t ea = cudaFuncSetAttribute(k_dense_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ea != cudaSuccess) return cuda_fail(ea, "cudaFuncSetAttribute(k_dense_sweep)");
  if (h.dense_inv) {
    ea = cudaFuncSetAttribute(k_dense_invert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dense_invert_smem(n, inv_w));
    if (ea != cudaSuccess) return cuda_fail(ea, "cudaFuncSetAttribute(k_dense_invert)");
  }
  cudaError_t e = cudaMalloc(&h.LU, bytes);
  if (e != cudaSuccess) {
    set_error("dense LU storage of " + std::to_string(bytes) + " bytes could not be allocated");
    return OCI_E_NOMEM;
  }
  e = cudaMalloc(&h.piv, (size_t)h.J * n * sizeof(int32_t));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(perm)");
  int *d_sing = nullptr;
  if ((e = cudaMalloc(&d_sing, sizeof(int))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  cudaMemsetAsync(d_sing, 0, sizeof(int), h.stream);
  k_dense_assemble<<<h.J, 256, 0, h.stream>>>(h.J, h.N, h.G, h.type, h.tt.dx, h.tt.sig, h.tt.Kap, h.v, h.dt, h.mu,
                                              h.w, h.LU);
  if (h.dense_inv)
    k_dense_invert<<<(h.J + inv_w - 1) / inv_w, inv_w * 32, dense_invert_smem(n, inv_w), h.stream>>>(
        h.J, n, h.LU, d_sing);
  else
    k_dense_factor<<<(h.J + 7) / 8, 256, 0, h.stream>>>(h.J, n, h.LU, h.piv, d_sing);
  int sing = 0;
  cudaMemcpyAsync(&sing, d_sing, sizeof(int), cudaMemcpyDeviceToHost, h.stream);
  e = cudaStreamSynchronize(h.stream);
  cudaFree(d_sing);
  if (e != cudaSuccess) return cuda_fail(e, "dense factorisation");
  if (sing) {
    set_error("a cell matrix A_j is singular");
    return OCI_E_SINGULAR;
  }
  return OCI_OK;
}

void launch_dense_step_const(Handle &h) {
  dim3 grid((h.J + 255) / 256, h.G * h.N);
  k_dense_step_const<<<grid, 256, 0, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.dx, h.v, h.dt, h.Q, h.psi_prev,
                                                 h.tc);
}

int dense_partials(const Handle &h) { return (h.J + kDenseWarps - 1) / kDenseWarps; }

void launch_dense_sweep(Handle &h) {
  const int n = 4 * h.N * h.G;
  if (h.dense_inv) {
    const size_t sm1 = (size_t)kDenseWarps * n * sizeof(double);
    const int nq = (n + 31) / 32;
#define OCI_DA(Q)                                                                                               \
  k_dense_apply<Q><<<dense_partials(h), kDenseWarps * 32, sm1, h.stream>>>(h.J, h.Jp, h.N, h.G, h.LU, h.mu, h.inc, \
                                                                          h.tc, h.Psi[0], h.Psi[1], h.ds, h.partials)
    if (nq <= 1) OCI_DA(1);
    else if (nq == 2) OCI_DA(2);
    else if (nq <= 4) OCI_DA(4);
    else OCI_DA(kDenseMaxNQ);
#undef OCI_DA
    return;
  }
  const size_t smem = (size_t)kDenseWarps * 2 * n * sizeof(double);
  k_dense_sweep<<<dense_partials(h), kDenseWarps * 32, smem, h.stream>>>(
      h.J, h.Jp, h.N, h.G, h.LU, h.piv, h.mu, h.inc, h.tc, h.Psi[0], h.Psi[1], h.ds, h.partials);
}

}  // namespace oci
