// oci_fourier.cu -- batched Fourier (von Neumann) analysis of the OCI and SI
// iterations (Sec. 2.3) on the GPU.
//
// Model problem: infinite homogeneous medium, one group, Sigma_t = v = 1, so a
// case (delta, tau, c) has dx = delta, dt = tau and Sigma_s = c; tau = +inf is
// the steady state.  A mode e^{i theta j} turns the lagged inflow of a cell into
// the neighbour's corner values times e^{-+ i theta}; with the cell operator L_c
// (Eq. Aj), the within-cell scattering S (Eq. scatter) and that inflow operator
// B(theta):
//   T_OCI(theta) = (L_c - S)^{-1} B(theta),    T_SI(theta) = (L_c - B(theta))^{-1} S.
// Both are reduced exactly to small matrices with the same nonzero spectrum:
//   - B has 2N nonzeros B[r_k, c_k] = f_k(theta) (mu > 0: rows kL, hL take kR, hR
//     of cell j-1 times mu e^{-i theta}; mu < 0: rows kR, hR take kL, hL of cell
//     j+1 times |mu| e^{i theta}), so B = U V^T with U = [f_k e_{r_k}],
//     V = [e_{c_k}], and the nonzero eigenvalues of T_OCI are those of
//     V^T (L_c - S)^{-1} U = C0 diag(f(theta)),  C0[k][l] = ((L_c - S)^{-1})[c_k][r_l],
//     a real, theta-independent 2N x 2N matrix (one FP64 solve per case);
//   - S = (delta c / 4) sum_p (1 (x) e_p)(w (x) e_p)^T has rank 4 and L_c - B is
//     block diagonal over the angles, so the nonzero eigenvalues of T_SI are those
//     of the 4 x 4 matrix  (delta c / 4) sum_n w_n (L_{c,n} - B_n(theta))^{-1}.
// The spectral radius of each small matrix M is lim ||M^n||^{1/n}, evaluated with
// 2^30 as n by normalised repeated squaring (Frobenius norm, FP64 complex);
// rho of a case is the maximum over theta_k = 2 pi k / (n_theta - 1).
// The time-march amplification of Sec. 2.2 (kind OCI_FOURIER_MARCH) is a 2x2
// matrix per ordinate in closed form; its eigenvalues come from the quadratic.
#include <math.h>

#include <vector>

#include "oci_internal.h"

namespace oci {
namespace {

struct cplx {
  double x, y;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx c) {
  return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
__device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }

constexpr int kSquarings = 30;
constexpr int kMaxFourierN = 32;

// 4x4 block of L_c for one ordinate (Eq. Aj with Sigma_t = v = 1).
__device__ __forceinline__ void lc_block(double mu, double delta, double alpha, double L[4][4]) {
  const double a = (fabs(mu) + delta) / 2.0;
  const double Lv[4][4] = {{a, mu / 2, alpha / 2, 0.0},
                           {-mu / 2, a, 0.0, alpha / 2},
                           {-alpha, 0.0, alpha + a, mu / 2},
                           {0.0, -alpha, -mu / 2, alpha + a}};
  for (int p = 0; p < 4; p++)
    for (int q = 0; q < 4; q++) L[p][q] = Lv[p][q];
}

// rows r_k (receiving) and columns c_k (neighbour corner) of the 2N nonzeros of B
__device__ __forceinline__ void b_entry(int k, int N, int &r, int &c) {
  const int m = k >> 1, h = k & 1;  // angle, (k or h corner pair)
  if (m >= N / 2) {                 // mu > 0 (ordinates ascending)
    r = 4 * m + 2 * h;
    c = r + 1;
  } else {
    r = 4 * m + 2 * h + 1;
    c = r - 1;
  }
}

// Per case: X = (L_c - S)^{-1} E_R by Gaussian elimination with partial pivoting
// on [A | E_R] in shared memory (A: n x n, E_R: the 2N unit columns r_l), then
// C0[k][l] = X[c_k][l].  One block per case.
__global__ void k_fourier_oci_setup(int N, const double *__restrict__ mu, const double *__restrict__ w,
                                    const double *__restrict__ delta, const double *__restrict__ tau,
                                    const double *__restrict__ cs, double *__restrict__ C0) {
  extern __shared__ double fs[];
  const int n = 4 * N, m2 = 2 * N, wdt = n + m2;
  double *A = fs;  // [n][wdt]
  __shared__ int piv;
  const int cse = blockIdx.x;
  const double d = delta[cse], t = tau[cse], c = cs[cse];
  const double alpha = isinf(t) ? 0.0 : d / t;
  for (int i = threadIdx.x; i < n * wdt; i += blockDim.x) A[i] = 0.0;
  __syncthreads();
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    double L[4][4];
    lc_block(mu[m], d, alpha, L);
    for (int p = 0; p < 4; p++)
      for (int q = 0; q < 4; q++) A[(4 * m + p) * wdt + 4 * m + q] = L[p][q];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N * N * 4; i += blockDim.x) {  // - S
    const int m = i / (4 * N), rem = i % (4 * N), nn = rem / 4, p = rem % 4;
    A[(4 * m + p) * wdt + 4 * nn + p] -= d * c / 4.0 * w[nn];
  }
  for (int l = threadIdx.x; l < m2; l += blockDim.x) {  // RHS unit columns e_{r_l}
    int r, cc;
    b_entry(l, N, r, cc);
    A[r * wdt + n + l] = 1.0;
  }
  __syncthreads();
  for (int k = 0; k < n; k++) {
    if (threadIdx.x == 0) {  // partial pivoting (first maximum)
      int best = k;
      double bv = fabs(A[k * wdt + k]);
      for (int i = k + 1; i < n; i++)
        if (fabs(A[i * wdt + k]) > bv) {
          bv = fabs(A[i * wdt + k]);
          best = i;
        }
      piv = best;
    }
    __syncthreads();
    if (piv != k)
      for (int j = threadIdx.x; j < wdt; j += blockDim.x) {
        const double tmp = A[k * wdt + j];
        A[k * wdt + j] = A[piv * wdt + j];
        A[piv * wdt + j] = tmp;
      }
    __syncthreads();
    const double inv = 1.0 / A[k * wdt + k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // eliminate column k in every other row
      if (i == k) continue;
      const double f = A[i * wdt + k] * inv;
      if (f != 0.0)
        for (int j = k; j < wdt; j++) A[i * wdt + j] -= f * A[k * wdt + j];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < wdt; j += blockDim.x)
      if (j != k) A[k * wdt + j] *= inv;
    __syncthreads();
    if (threadIdx.x == 0) A[k * wdt + k] = 1.0;
    __syncthreads();
  }
  double *out = C0 + (size_t)cse * m2 * m2;
  for (int i = threadIdx.x; i < m2 * m2; i += blockDim.x) {
    const int k = i / m2, l = i % m2;
    int r, cc;
    b_entry(k, N, r, cc);
    out[i] = A[cc * wdt + n + l];
  }
}

// Spectral radius of the m x m complex matrix in M (shared memory, row-major)
// by normalised repeated squaring; scratch P of the same size.  Whole block.
__device__ double spectral_radius_sq(cplx *M, cplx *P, int m, double *red) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  double logn = 0.0;  // log ||T^(2^s)|| so far
  for (int s = 0; s <= kSquarings; s++) {
    // Frobenius norm (fixed order), normalise
    double v = 0.0;
    for (int i = tid; i < m * m; i += nthr) v += cabs2(M[i]);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < (nthr + 31) / 32; i++) tot += red[i];
      red[32] = tot;
    }
    __syncthreads();
    const double nrm = sqrt(red[32]);
    if (isnan(nrm)) return nrm;          // non-finite input
    if (!(nrm > 0.0)) return 0.0;        // nilpotent: rho = 0
    // M currently holds T^(2^s) / exp(logn_prev): its norm contributes at this power
    logn += log(nrm);
    if (s == kSquarings) break;
    const double inv = 1.0 / nrm;
    for (int i = tid; i < m * m; i += nthr) {
      M[i].x *= inv;
      M[i].y *= inv;
    }
    __syncthreads();
    for (int i = tid; i < m * m; i += nthr) {  // P = M * M
      const int r = i / m, c = i % m;
      cplx acc = {0.0, 0.0};
      for (int k = 0; k < m; k++) acc = cfma(M[r * m + k], M[k * m + c], acc);
      P[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < m * m; i += nthr) M[i] = P[i];
    __syncthreads();
    logn *= 2.0;  // (T^(2^s))^2 = T^(2^(s+1)); the new product's norm is added next pass
  }
  return exp(logn / ldexp(1.0, kSquarings));
}

__device__ __forceinline__ void atomic_max_pos(double *addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// One block per (theta, case): rho of C0 diag(f(theta)).
__global__ void k_fourier_rho_oci(int N, int n_theta, const double *__restrict__ mu,
                                  const double *__restrict__ C0, double *__restrict__ rho) {
  extern __shared__ double fs[];
  __shared__ double red[33];
  const int m2 = 2 * N;
  cplx *M = (cplx *)fs, *P = M + m2 * m2;
  const int it = blockIdx.x, cse = blockIdx.y;
  const double th = n_theta > 1 ? 2.0 * M_PI * it / (n_theta - 1) : 0.0;
  const double *c0 = C0 + (size_t)cse * m2 * m2;
  for (int i = threadIdx.x; i < m2 * m2; i += blockDim.x) {
    const int l = i % m2, ang = l >> 1;
    const double mm = mu[ang];
    // f_l = mu e^{-i theta} (mu > 0), |mu| e^{+i theta} (mu < 0)
    const cplx f = mm > 0 ? cplx{mm * cos(th), -mm * sin(th)} : cplx{-mm * cos(th), -mm * sin(th)};
    M[i] = {c0[i] * f.x, c0[i] * f.y};
  }
  __syncthreads();
  const double r = spectral_radius_sq(M, P, m2, red);
  if (threadIdx.x == 0) atomic_max_pos(rho + cse, r);
}

// 4x4 complex inverse by Gauss-Jordan with partial pivoting (one thread).
__device__ bool inv4(cplx A[4][4], cplx X[4][4]) {
  for (int p = 0; p < 4; p++)
    for (int q = 0; q < 4; q++) X[p][q] = {p == q ? 1.0 : 0.0, 0.0};
  for (int k = 0; k < 4; k++) {
    int b = k;
    for (int i = k + 1; i < 4; i++)
      if (cabs2(A[i][k]) > cabs2(A[b][k])) b = i;
    if (cabs2(A[b][k]) == 0.0) return false;
    if (b != k)
      for (int j = 0; j < 4; j++) {
        cplx t = A[k][j];
        A[k][j] = A[b][j];
        A[b][j] = t;
        t = X[k][j];
        X[k][j] = X[b][j];
        X[b][j] = t;
      }
    const double d2 = cabs2(A[k][k]);
    const cplx inv = {A[k][k].x / d2, -A[k][k].y / d2};
    for (int j = 0; j < 4; j++) {
      A[k][j] = cmul(A[k][j], inv);
      X[k][j] = cmul(X[k][j], inv);
    }
    for (int i = 0; i < 4; i++) {
      if (i == k) continue;
      const cplx f = A[i][k];
      for (int j = 0; j < 4; j++) {
        A[i][j] = cfma({-f.x, -f.y}, A[k][j], A[i][j]);
        X[i][j] = cfma({-f.x, -f.y}, X[k][j], X[i][j]);
      }
    }
  }
  return true;
}

// One warp per (theta, case): K = (delta c / 4) sum_n w_n (L_{c,n} - B_n)^{-1}, rho(K).
__global__ void k_fourier_rho_si(int N, int n_theta, const double *__restrict__ mu, const double *__restrict__ w,
                                 const double *__restrict__ delta, const double *__restrict__ tau,
                                 const double *__restrict__ cs, double *__restrict__ rho) {
  __shared__ cplx Ks[16], Ps[16];
  __shared__ double red[33];
  const int it = blockIdx.x, cse = blockIdx.y, lane = threadIdx.x;
  const double th = n_theta > 1 ? 2.0 * M_PI * it / (n_theta - 1) : 0.0;
  const double d = delta[cse], t = tau[cse], c = cs[cse];
  const double alpha = isinf(t) ? 0.0 : d / t;
  cplx acc[16];
  for (int i = 0; i < 16; i++) acc[i] = {0.0, 0.0};
  bool ok = true;
  for (int n = lane; n < N; n += 32) {
    double L[4][4];
    lc_block(mu[n], d, alpha, L);
    cplx A[4][4], X[4][4];
    for (int p = 0; p < 4; p++)
      for (int q = 0; q < 4; q++) A[p][q] = {L[p][q], 0.0};
    if (mu[n] > 0) {  // - B_n: rows kL, hL take the R corners of cell j-1
      const cplx f = {mu[n] * cos(th), -mu[n] * sin(th)};
      A[0][1] = {A[0][1].x - f.x, A[0][1].y - f.y};
      A[2][3] = {A[2][3].x - f.x, A[2][3].y - f.y};
    } else {
      const cplx f = {-mu[n] * cos(th), -mu[n] * sin(th)};
      A[1][0] = {A[1][0].x - f.x, A[1][0].y - f.y};
      A[3][2] = {A[3][2].x - f.x, A[3][2].y - f.y};
    }
    ok = ok && inv4(A, X);
    for (int p = 0; p < 4; p++)
      for (int q = 0; q < 4; q++) {
        acc[p * 4 + q].x += w[n] * X[p][q].x;
        acc[p * 4 + q].y += w[n] * X[p][q].y;
      }
  }
  for (int i = 0; i < 16; i++)
    for (int o = 16; o > 0; o >>= 1) {
      acc[i].x += __shfl_down_sync(0xffffffffu, acc[i].x, o);
      acc[i].y += __shfl_down_sync(0xffffffffu, acc[i].y, o);
    }
  const bool all_ok = __all_sync(0xffffffffu, ok);
  if (lane == 0)
    for (int i = 0; i < 16; i++) Ks[i] = {acc[i].x * d * c / 4.0, acc[i].y * d * c / 4.0};
  __syncwarp();
  const double r = all_ok ? spectral_radius_sq(Ks, Ps, 4, red) : INFINITY;
  if (lane == 0) atomic_max_pos(rho + cse, r);
}

__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  const double d = cabs2(b);
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// Principal square root of a complex number (half-angle form).
__device__ __forceinline__ cplx csqrt_(cplx z) {
  const double r = hypot(z.x, z.y);
  const double re = sqrt(fmax(0.0, 0.5 * (r + z.x)));
  const double im = sqrt(fmax(0.0, 0.5 * (r - z.x)));
  return {re, z.y < 0.0 ? -im : im};
}

// Time-march amplification of Sec. 2.2 (infinite homogeneous medium, no
// scattering, Sigma = v = 1 so dx = delta and dt = tau): per ordinate and wave
// number the 2x2 matrix K = gamma (K+- K+- + (dx/(v dt)) K+- + gamma I)^{-1},
// gamma = (dx/(v dt)) (dx/(2 v dt)), with
//   K+ = [[mu/2 + delta/2, mu (1/2 - e^{-i theta})], [-mu/2, mu/2 + delta/2]]     (mu > 0)
//   K- = [[-mu/2 + delta/2, mu/2], [mu (e^{i theta} - 1/2), -mu/2 + delta/2]]     (mu < 0)
// and its eigenvalues from the characteristic quadratic.  One thread per
// (theta, ordinate, case); rho of a case = the largest |lambda| over all of them.
__global__ void k_fourier_rho_march(int N, int n_theta, int n_cases, const double *__restrict__ mu,
                                    const double *__restrict__ delta, const double *__restrict__ tau,
                                    double *__restrict__ rho) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n_theta * N * n_cases;
  if (gid >= total) return;
  const int cse = (int)(gid / ((long long)n_theta * N));
  const int rem = (int)(gid % ((long long)n_theta * N));
  const int it = rem / N, m = rem % N;
  const double d = delta[cse], t = tau[cse];
  if (isinf(t)) {  // steady state: no time march (K = 0)
    atomic_max_pos(rho + cse, 0.0);
    return;
  }
  const double th = n_theta > 1 ? 2.0 * M_PI * it / (n_theta - 1) : 0.0;
  const double mm = mu[m], al = d / t, g = al * al / 2.0;
  const double cs = cos(th), sn = sin(th);
  cplx k00, k01, k10, k11;
  if (mm > 0) {
    k00 = {mm / 2 + d / 2, 0.0};
    k01 = {mm * (0.5 - cs), mm * sn};  // mu (1/2 - e^{-i theta})
    k10 = {-mm / 2, 0.0};
    k11 = k00;
  } else {
    k00 = {-mm / 2 + d / 2, 0.0};
    k01 = {mm / 2, 0.0};
    k10 = {mm * (cs - 0.5), mm * sn};  // mu (e^{i theta} - 1/2)
    k11 = k00;
  }
  // Q = K K + al K + g I
  const cplx q00 = {cmul(k00, k00).x + cmul(k01, k10).x + al * k00.x + g, cmul(k00, k00).y + cmul(k01, k10).y + al * k00.y};
  const cplx q01 = {cmul(k00, k01).x + cmul(k01, k11).x + al * k01.x, cmul(k00, k01).y + cmul(k01, k11).y + al * k01.y};
  const cplx q10 = {cmul(k10, k00).x + cmul(k11, k10).x + al * k10.x, cmul(k10, k00).y + cmul(k11, k10).y + al * k10.y};
  const cplx q11 = {cmul(k10, k01).x + cmul(k11, k11).x + al * k11.x + g, cmul(k10, k01).y + cmul(k11, k11).y + al * k11.y};
  // K = g Q^{-1} = g / det(Q) [[q11, -q01], [-q10, q00]]
  const cplx det = {cmul(q00, q11).x - cmul(q01, q10).x, cmul(q00, q11).y - cmul(q01, q10).y};
  const cplx sc = cdiv({g, 0.0}, det);
  const cplx a = cmul(sc, q11), b = cmul(sc, {-q01.x, -q01.y}), c = cmul(sc, {-q10.x, -q10.y}), e = cmul(sc, q00);
  // eigenvalues of [[a, b], [c, e]]: (tr +- sqrt(tr^2 - 4 det)) / 2
  const cplx tr = {a.x + e.x, a.y + e.y};
  const cplx dk = {cmul(a, e).x - cmul(b, c).x, cmul(a, e).y - cmul(b, c).y};
  const cplx disc = csqrt_({cmul(tr, tr).x - 4.0 * dk.x, cmul(tr, tr).y - 4.0 * dk.y});
  const cplx l1 = {0.5 * (tr.x + disc.x), 0.5 * (tr.y + disc.y)};
  const cplx l2 = {0.5 * (tr.x - disc.x), 0.5 * (tr.y - disc.y)};
  const double r = fmax(sqrt(cabs2(l1)), sqrt(cabs2(l2)));
  atomic_max_pos(rho + cse, isfinite(r) ? r : INFINITY);
}

bool is_dev(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace oci

using namespace oci;

extern "C" int oci_fourier_rho(int32_t kind, int32_t N, int32_t n_cases, const double *delta, const double *tau,
                               const double *c, int32_t n_theta, double *rho, void *stream) {
  if (kind != OCI_FOURIER_OCI && kind != OCI_FOURIER_SI && kind != OCI_FOURIER_MARCH)
    return set_error("kind must be OCI_FOURIER_OCI, _SI or _MARCH"), OCI_E_INVAL;
  const bool march = kind == OCI_FOURIER_MARCH;
  if (N < 2 || N > kMaxFourierN || (N & 1)) return set_error("N must be even, 2 <= N <= 32"), OCI_E_INVAL;
  if (n_cases < 1 || n_theta < 1 || n_cases > 65535)
    return set_error("need 1 <= n_cases <= 65535 and n_theta >= 1"), OCI_E_INVAL;
  if (march && ((long long)n_theta * N * n_cases + 255) / 256 > 2147483647LL)
    return set_error("n_theta * N * n_cases too large for one launch"), OCI_E_INVAL;
  if (!delta || !tau || (!c && !march) || !rho) return set_error("delta, tau, c and rho must be given"), OCI_E_INVAL;
  const bool dev_in = is_dev(delta);
  if (dev_in != is_dev(tau) || (c && dev_in != is_dev(c)))
    return set_error("delta, tau, c: all host or all device"), OCI_E_INVAL;
  std::vector<double> hd(n_cases), ht(n_cases), hc(n_cases);
  cudaStream_t st = (cudaStream_t)stream;
  if (dev_in) {
    cudaMemcpy(hd.data(), delta, n_cases * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(ht.data(), tau, n_cases * 8, cudaMemcpyDeviceToHost);
    if (c) cudaMemcpy(hc.data(), c, n_cases * 8, cudaMemcpyDeviceToHost);
  } else {
    hd.assign(delta, delta + n_cases);
    ht.assign(tau, tau + n_cases);
    if (c) hc.assign(c, c + n_cases);
  }
  if (march) hc.assign(n_cases, 0.0);  // the time-march model problem has no scattering
  for (int i = 0; i < n_cases; i++)
    if (!(hd[i] > 0.0) || !isfinite(hd[i]) || !(ht[i] > 0.0) || !(hc[i] >= 0.0) || !isfinite(hc[i]))
      return set_error("each case needs delta > 0 finite, tau > 0 (inf: steady state), c >= 0"), OCI_E_INVAL;
  std::vector<double> mu, w;
  gauss_legendre(N, mu, w);
  const int m2 = 2 * N, n = 4 * N;
  double *dbuf = nullptr;
  const size_t nb = 2 * (size_t)N + 4 * (size_t)n_cases + (size_t)n_cases * m2 * m2;
  cudaError_t e = cudaMalloc(&dbuf, nb * 8);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(Fourier scratch)");
  double *d_mu = dbuf, *d_w = d_mu + N, *d_del = d_w + N, *d_tau = d_del + n_cases, *d_c = d_tau + n_cases,
         *d_rho = d_c + n_cases, *d_C0 = d_rho + n_cases;
  int rc = OCI_OK;
  do {
    if ((e = cudaMemcpyAsync(d_mu, mu.data(), N * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d_w, w.data(), N * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d_del, hd.data(), n_cases * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d_tau, ht.data(), n_cases * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d_c, hc.data(), n_cases * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(d_rho, 0, n_cases * 8, st)) != cudaSuccess) break;
    if (kind == OCI_FOURIER_OCI) {
      const size_t sm1 = (size_t)n * (n + m2) * 8;
      if ((e = cudaFuncSetAttribute(k_fourier_oci_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1)) !=
          cudaSuccess)
        break;
      k_fourier_oci_setup<<<n_cases, 256, sm1, st>>>(N, d_mu, d_w, d_del, d_tau, d_c, d_C0);
      const size_t sm2 = (size_t)2 * m2 * m2 * sizeof(double) * 2;
      if ((e = cudaFuncSetAttribute(k_fourier_rho_oci, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) !=
          cudaSuccess)
        break;
      k_fourier_rho_oci<<<dim3(n_theta, n_cases), 256, sm2, st>>>(N, n_theta, d_mu, d_C0, d_rho);
    } else if (kind == OCI_FOURIER_SI) {
      k_fourier_rho_si<<<dim3(n_theta, n_cases), 32, 0, st>>>(N, n_theta, d_mu, d_w, d_del, d_tau, d_c, d_rho);
    } else {
      const long long total = (long long)n_theta * N * n_cases;
      k_fourier_rho_march<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(N, n_theta, n_cases, d_mu, d_del, d_tau,
                                                                           d_rho);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(rho, d_rho, n_cases * 8, cudaMemcpyDefault, st)) != cudaSuccess) break;
    e = cudaStreamSynchronize(st);
  } while (false);
  if (e != cudaSuccess) rc = cuda_fail(e, "oci_fourier_rho");
  cudaFree(dbuf);
  return rc;
}
