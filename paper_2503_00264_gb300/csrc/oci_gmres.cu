// oci_gmres.cu -- Krylov (GMRES) acceleration of the FP64 OCI time step.
//
// One OCI sweep is the affine map F(x) = T x + b with T = A^{-1} B (the lagged
// inflow through the cell solves, Eq. oci) and b = A^{-1}(c + incident flux):
// plain OCI is the fixed-point iteration x <- F(x).  The same fixed point solves
// the linear system (I - T) x = b, which restarted GMRES(m) solves with one
// sweep per Krylov vector (T v = a sweep of v with zero constant and zero
// incident flux).  The residual b - (I - T) x = F(x) - x is exactly the change
// one OCI sweep would make from x, i.e. the e of Sec. 2.1 at x; the step ends
// when it falls below tol times a factor (the caller's; the plain rule
// e < tol (1 - rho) bounds the error by about tol, and ||x - x*|| <= ||r|| /
// (1 - rho) for GMRES), and the committed iterate is F(x), so the step's last
// operation is an OCI sweep as in the plain form.  Orthogonalisation: classical
// Gram-Schmidt applied twice; the dot products of a pass are one kernel reading
// w and the basis once, summed in a fixed order (bit-reproducible).  The small
// Hessenberg least-squares problem is solved on the host with Givens rotations.
#include <math.h>

#include <algorithm>
#include <vector>

#include "oci_internal.h"

namespace oci {
namespace {

constexpr int kGmMaxK = 33;  // basis vectors (restart length + 1)
constexpr int kGmThreads = 256;

// part[i][block] = sum over the block's elements of V_i . w, i < k (fixed order)
__global__ void __launch_bounds__(kGmThreads) k_gm_mdot(const double *__restrict__ V, size_t ld, int k,
                                                         const double *__restrict__ w, size_t n, size_t chunk,
                                                         double *__restrict__ part) {
  __shared__ double red[kGmThreads / 32][kGmMaxK];
  const size_t e0 = (size_t)blockIdx.x * chunk, e1 = min(n, e0 + chunk);
  double acc[kGmMaxK];
#pragma unroll
  for (int i = 0; i < kGmMaxK; i++) acc[i] = 0.0;
  for (size_t e = e0 + threadIdx.x; e < e1; e += kGmThreads) {
    const double we = w[e];
#pragma unroll
    for (int i = 0; i < kGmMaxK; i++)
      if (i < k) acc[i] = fma(V[(size_t)i * ld + e], we, acc[i]);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kGmMaxK; i++) {
    if (i >= k) break;
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += kGmThreads) {
    double s = 0.0;
    for (int q = 0; q < kGmThreads / 32; q++) s += red[q][i];
    part[(size_t)i * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_gm_sum(const double *__restrict__ part, int nb, int k, double *__restrict__ out) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[(size_t)i * nb + b];
    out[i] = s;
  }
}

// w += sign * sum_i c[i] V_i
__global__ void k_gm_maxpy(double *__restrict__ w, const double *__restrict__ V, size_t ld, int k,
                           const double *__restrict__ c, double sign, size_t n) {
  __shared__ double cs[kGmMaxK];
  if (threadIdx.x < k) cs[threadIdx.x] = sign * c[threadIdx.x];
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = w[e];
    for (int i = 0; i < k; i++) v = fma(cs[i], V[(size_t)i * ld + e], v);
    w[e] = v;
  }
}

// z = a x + b y
__global__ void k_gm_axpby(double *__restrict__ z, double a, const double *__restrict__ x, double b,
                           const double *__restrict__ y, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    z[e] = a * x[e] + b * y[e];
}

struct Gm {
  Handle &h;
  size_t n, chunk;
  int nb, grid;
  Gm(Handle &hh) : h(hh) {
    n = (size_t)h.G * h.N * 4 * h.Jp;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    nb = 4 * sms;
    chunk = (n + nb - 1) / nb;
    grid = 4 * sms;
  }
  double *V(int i) { return h.gm_V + (size_t)i * n; }
  // h_out[0:k) = V_i . w (device, then host)
  int dots(int k, const double *w, const double *Vb, std::vector<double> &out) {
    k_gm_mdot<<<nb, kGmThreads, 0, h.stream>>>(Vb, n, k, w, n, chunk, h.gm_part);
    k_gm_sum<<<1, 64, 0, h.stream>>>(h.gm_part, nb, k, h.gm_h);
    out.resize(k);
    cudaError_t e = cudaMemcpyAsync(out.data(), h.gm_h, k * 8, cudaMemcpyDeviceToHost, h.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h.stream);
    if (e != cudaSuccess) return cuda_fail(e, "GMRES dot products");
    return OCI_OK;
  }
  int norm(const double *w, double &out) {
    std::vector<double> v;
    int rc = dots(1, w, w, v);
    out = rc ? 0.0 : sqrt(v[0]);
    return rc;
  }
  int maxpy(double *w, int k, const std::vector<double> &c, double sign) {
    cudaError_t e = cudaMemcpyAsync(h.gm_h, c.data(), k * 8, cudaMemcpyHostToDevice, h.stream);
    if (e != cudaSuccess) return cuda_fail(e, "GMRES coefficients");
    k_gm_maxpy<<<grid, kGmThreads, 0, h.stream>>>(w, h.gm_V, n, k, h.gm_h, sign, n);
    return OCI_OK;
  }
  void axpby(double *z, double a, const double *x, double b, const double *y) {
    k_gm_axpby<<<grid, kGmThreads, 0, h.stream>>>(z, a, x, b, y, n);
  }
};

}  // namespace

int gmres_alloc(Handle &h) {
  if (h.gm_V) return OCI_OK;
  const size_t n = (size_t)h.G * h.N * 4 * h.Jp;
  const int m = h.gm_restart;
  const size_t K = 2 * (size_t)h.G * h.N * 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if ((e = cudaMalloc(&h.gm_V, (size_t)(m + 1) * n * 8)) != cudaSuccess ||
      (e = cudaMalloc(&h.gm_w, 2 * n * 8)) != cudaSuccess || (e = cudaMalloc(&h.gm_zero, (n + K) * 8)) != cudaSuccess ||
      (e = cudaMalloc(&h.gm_part, (size_t)kGmMaxK * 4 * sms * 8)) != cudaSuccess ||
      (e = cudaMalloc(&h.gm_h, kGmMaxK * 8)) != cudaSuccess || (e = cudaMalloc(&h.gm_ds, sizeof(DevState))) != cudaSuccess)
    return cuda_fail(e, "GMRES storage");
  // zero padding columns everywhere: every vector stays zero there
  if ((e = cudaMemsetAsync(h.gm_V, 0, (size_t)(m + 1) * n * 8, h.stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(h.gm_w, 0, 2 * n * 8, h.stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(h.gm_zero, 0, (n + K) * 8, h.stream)) != cudaSuccess)
    return cuda_fail(e, "GMRES storage");
  DevState d;
  memset(&d, 0, sizeof d);
  d.fixed = 1;
  if ((e = cudaMemcpyAsync(h.gm_ds, &d, sizeof d, cudaMemcpyHostToDevice, h.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h.stream)) != cudaSuccess)
    return cuda_fail(e, "GMRES storage");
  return OCI_OK;
}

void gmres_free(Handle &h) {
  void *ps[] = {h.gm_V, h.gm_w, h.gm_zero, h.gm_part, h.gm_h, h.gm_ds};
  for (void *p : ps)
    if (p) cudaFree(p);
  h.gm_V = h.gm_w = h.gm_zero = h.gm_part = h.gm_h = nullptr;
  h.gm_ds = nullptr;
}

// One time step by GMRES(m) on (I - T) x = b from x0 = Psi[cur]; on return
// Psi[cur] holds F(x) and the host state record the outcome (l = sweeps).
int gmres_solve(Handle &h, double tol_g, int max_sweeps, int &sweeps, double &e_last, int &status) {
  int rc = gmres_alloc(h);
  if (rc) return rc;
  Gm g(h);
  const int m = h.gm_restart;
  double *x = h.Psi[h.h_ds->cur];
  double *Fx = h.gm_w;      // F(x) or T v
  double *w = h.gm_w + g.n;  // Arnoldi vector
  const double *tc0 = h.gm_zero, *inc0 = h.gm_zero + g.n;
  sweeps = 0;
  status = OCI_E_NOCONV;
  e_last = 0.0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hc, hc2, y;
  for (;;) {
    launch_oci_apply(h, x, Fx, h.tc, h.inc, h.gm_ds);  // F(x)
    sweeps++;
    g.axpby(g.V(0), 1.0, Fx, -1.0, x);  // r = F(x) - x
    double beta;
    if ((rc = g.norm(g.V(0), beta))) return rc;
    e_last = beta;
    if (!std::isfinite(beta)) {
      status = OCI_E_NONFINITE;
      break;
    }
    if (beta < tol_g) {
      status = OCI_OK;
      break;
    }
    if (sweeps >= max_sweeps) break;
    g.axpby(g.V(0), 1.0 / beta, g.V(0), 0.0, g.V(0));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jl = -1;
    for (int j = 0; j < m; j++) {
      launch_oci_apply(h, g.V(j), Fx, tc0, inc0, h.gm_ds);  // T V_j
      sweeps++;
      g.axpby(w, 1.0, g.V(j), -1.0, Fx);  // w = (I - T) V_j
      if ((rc = g.dots(j + 1, w, h.gm_V, hc))) return rc;
      if ((rc = g.maxpy(w, j + 1, hc, -1.0))) return rc;
      if ((rc = g.dots(j + 1, w, h.gm_V, hc2))) return rc;  // second pass
      if ((rc = g.maxpy(w, j + 1, hc2, -1.0))) return rc;
      for (int i = 0; i <= j; i++) hc[i] += hc2[i];
      double hn;
      if ((rc = g.norm(w, hn))) return rc;
      if (hn > 0.0) g.axpby(g.V(j + 1), 1.0 / hn, w, 0.0, w);
      // Givens: previous rotations on column j, then a new one zeroing H[j+1][j]
      for (int i = 0; i < j; i++) {
        const double a = hc[i], b = hc[i + 1];
        hc[i] = cs[i] * a + sn[i] * b;
        hc[i + 1] = -sn[i] * a + cs[i] * b;
      }
      const double a = hc[j], b = hn, r = hypot(a, b);
      cs[j] = r > 0.0 ? a / r : 1.0;
      sn[j] = r > 0.0 ? b / r : 0.0;
      hc[j] = r;
      for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = hc[i];
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      jl = j;
      if (fabs(gv[j + 1]) < tol_g || sweeps >= max_sweeps || !(hn > 0.0)) break;
    }
    // y = H^{-1} g (upper triangular, jl + 1 unknowns); x += V y
    y.assign(jl + 1, 0.0);
    for (int i = jl; i >= 0; i--) {
      double v = gv[i];
      for (int k = i + 1; k <= jl; k++) v -= H[(size_t)i * m + k] * y[k];
      y[i] = v / H[(size_t)i * m + i];
    }
    if ((rc = g.maxpy(x, jl + 1, y, 1.0))) return rc;
  }
  // commit F(x): the last operation of the step is an OCI sweep
  cudaError_t e = cudaMemcpyAsync(x, Fx, g.n * 8, cudaMemcpyDeviceToDevice, h.stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "GMRES step");
  return OCI_OK;
}

}  // namespace oci
