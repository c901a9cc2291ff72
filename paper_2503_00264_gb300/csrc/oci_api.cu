// oci_api.cu -- the C ABI of liboci (include/oci.h): validation, setup of the
// per-cell-type tables, device state, the convergence loops as CUDA graphs with a
// conditional WHILE node, and state access.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "oci_internal.h"


namespace oci {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return OCI_E_CUDA;
}

int si_partials(const Handle &h);
int dense_partials(const Handle &h);
void launch_si_phi_from_psi(Handle &h, double *);
void launch_mx_settle(Handle &h, int kind);
const void *k_mx_inner_ptr();

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

// ---------------------------------------------------------------- quadrature
// Gauss-Legendre nodes/weights on [-1,1] (the paper uses Gauss-Legendre S_N
// throughout, Sec. 1): Newton iteration on P_N from Tricomi's initial guess;
// P_N and P_N' from the three-term recurrence.  Ascending nodes.
void gauss_legendre(int N, std::vector<double> &x, std::vector<double> &wt) {
  x.assign(N, 0.0);
  wt.assign(N, 0.0);
  const double pi = 3.141592653589793238462643;
  for (int k = 1; k <= (N + 1) / 2; k++) {
    double z = (1.0 - 1.0 / (8.0 * N * N) + 1.0 / (8.0 * N * N * N)) * cos(pi * (4.0 * k - 1.0) / (4.0 * N + 2.0));
    double dP = 1.0;
    for (int it = 0; it < 100; it++) {
      double pm1 = 1.0, p = z;
      for (int n = 1; n < N; n++) {
        const double pn = ((2.0 * n + 1.0) * z * p - n * pm1) / (n + 1.0);
        pm1 = p;
        p = pn;
      }
      dP = N * (pm1 - z * p) / (1.0 - z * z);
      const double dz = p / dP;
      z -= dz;
      if (fabs(dz) <= 1e-17) break;
    }
    {
      double pm1 = 1.0, p = z;
      for (int n = 1; n < N; n++) {
        const double pn = ((2.0 * n + 1.0) * z * p - n * pm1) / (n + 1.0);
        pm1 = p;
        p = pn;
      }
      dP = N * (pm1 - z * p) / (1.0 - z * z);
    }
    const double wk = 2.0 / ((1.0 - z * z) * dP * dP);
    x[N - k] = z;       // k-th largest node
    x[k - 1] = -z;
    wt[N - k] = wk;
    wt[k - 1] = wk;
  }
}

// Dense inverse by Gauss-Jordan elimination with partial pivoting (host, FP64).
static bool invert(int n, std::vector<double> A, std::vector<double> &inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) inv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; k++) {
    int pr = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int r = k + 1; r < n; r++)
      if (fabs(A[(size_t)r * n + k]) > best) {
        best = fabs(A[(size_t)r * n + k]);
        pr = r;
      }
    if (best == 0.0 || !std::isfinite(best)) return false;
    if (pr != k)
      for (int c = 0; c < n; c++) {
        std::swap(A[(size_t)k * n + c], A[(size_t)pr * n + c]);
        std::swap(inv[(size_t)k * n + c], inv[(size_t)pr * n + c]);
      }
    const double d = A[(size_t)k * n + k];
    for (int c = 0; c < n; c++) {
      A[(size_t)k * n + c] /= d;
      inv[(size_t)k * n + c] /= d;
    }
    for (int r = 0; r < n; r++) {
      if (r == k) continue;
      const double f = A[(size_t)r * n + k];
      if (f == 0.0) continue;
      for (int c = 0; c < n; c++) {
        A[(size_t)r * n + c] -= f * A[(size_t)k * n + c];
        inv[(size_t)r * n + c] -= f * inv[(size_t)k * n + c];
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------- validation
static bool finite_ge(const double *a, size_t n, double lo, bool strict) {
  for (size_t i = 0; i < n; i++) {
    if (!std::isfinite(a[i])) return false;
    if (strict ? !(a[i] > lo) : !(a[i] >= lo)) return false;
  }
  return true;
}
static bool all_finite(const double *a, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(a[i])) return false;
  return true;
}

int validate(const oci_problem *p) {
  if (!p) return set_error("problem is NULL"), OCI_E_INVAL;
  if (p->J < 1) return set_error("J must be >= 1"), OCI_E_INVAL;
  if (p->N < 2 || p->N > kMaxN || (p->N & 1)) return set_error("N must be even, 2 <= N <= 128"), OCI_E_INVAL;
  if (p->G < 1 || p->G > kMaxG) return set_error("G must be in [1, 16]"), OCI_E_INVAL;
  if (4 * p->N * p->G > kMaxUnknowns) return set_error("4*N*G must be <= 2048"), OCI_E_INVAL;
  if (p->n_mat < 1) return set_error("n_mat must be >= 1"), OCI_E_INVAL;
  if (!p->dx || !p->mat || !p->sigma_t || !p->sigma_s || !p->v)
    return set_error("dx, mat, sigma_t, sigma_s and v are required"), OCI_E_INVAL;
  const size_t J = p->J, G = p->G, N = p->N, M = p->n_mat;
  if (!finite_ge(p->dx, J, 0.0, true)) return set_error("dx must be finite and > 0"), OCI_E_INVAL;
  for (size_t j = 0; j < J; j++)
    if (p->mat[j] < 0 || p->mat[j] >= p->n_mat) return set_error("mat out of range"), OCI_E_INVAL;
  if (!finite_ge(p->sigma_t, M * G, 0.0, false)) return set_error("sigma_t must be finite and >= 0"), OCI_E_INVAL;
  if (!finite_ge(p->sigma_s, M * G * G, 0.0, false)) return set_error("sigma_s must be finite and >= 0"), OCI_E_INVAL;
  if (!finite_ge(p->v, G, 0.0, true)) return set_error("v must be finite and > 0"), OCI_E_INVAL;
  if (!(std::isfinite(p->dt) && p->dt > 0)) return set_error("dt must be finite and > 0"), OCI_E_INVAL;
  if (p->Q && !all_finite(p->Q, J * G * 4)) return set_error("Q must be finite"), OCI_E_INVAL;
  if (p->psi_init && !all_finite(p->psi_init, J * G * N * 2)) return set_error("psi_init must be finite"), OCI_E_INVAL;
  if (p->inc_left && !all_finite(p->inc_left, G * N * 2)) return set_error("inc_left must be finite"), OCI_E_INVAL;
  if (p->inc_right && !all_finite(p->inc_right, G * N * 2)) return set_error("inc_right must be finite"), OCI_E_INVAL;
  if (!(std::isfinite(p->tol) && p->tol >= 0)) return set_error("tol must be finite and >= 0"), OCI_E_INVAL;
  if (p->max_iter < 1) return set_error("max_iter must be >= 1"), OCI_E_INVAL;
  if (p->precision < OCI_FP64 || p->precision > OCI_FP32_IR) return set_error("bad precision"), OCI_E_INVAL;
  if (p->guess < OCI_GUESS_PREV || p->guess > OCI_GUESS_USER) return set_error("bad guess policy"), OCI_E_INVAL;
  if (p->solver < OCI_SOLVER_AUTO || p->solver > OCI_SOLVER_DENSE_LU) return set_error("bad solver"), OCI_E_INVAL;
  if (p->precision != OCI_FP64 && p->solver == OCI_SOLVER_DENSE_LU)
    return set_error("the dense per-cell solver is FP64 only"), OCI_E_INVAL;
  if (p->solver == OCI_SOLVER_DENSE_LU && 4 * p->N * p->G > 1024)
    return set_error("the dense per-cell solver needs 4*N*G <= 1024"), OCI_E_INVAL;
  if ((p->precision == OCI_TF32_IR || p->precision == OCI_BF16X3_IR) &&
      (4 * p->N * p->G > 512 || (4 * p->N * p->G) % 32 != 0))
    return set_error("the tensor-core forms need 4*N*G <= 512 and a multiple of 32"), OCI_E_INVAL;
  return OCI_OK;
}

// ---------------------------------------------------------------- tables
// Per unique (material, dx) cell type: L_{g,m}^{-1} (Eq. Aj), the inflow columns,
// Mp = (I - K H)^{-1} K and K.
int build_tables(Handle &h, std::vector<double> &Linv, std::vector<double> &Cin, std::vector<double> &Mp,
                 std::vector<double> &Kap, std::vector<double> &tdx, std::vector<double> &tsig,
                 std::vector<double> &Lco) {
  const int N = h.N, G = h.G, J = h.J;
  std::map<std::pair<int, uint64_t>, int> ids;
  h.h_type.assign(J, 0);
  std::vector<std::pair<int, double>> types;
  for (int j = 0; j < J; j++) {
    uint64_t bits;
    std::memcpy(&bits, &h.h_dx[j], 8);
    auto key = std::make_pair((int)h.h_mat[j], bits);
    auto it = ids.find(key);
    if (it == ids.end()) {
      const int id = (int)types.size();
      ids.emplace(key, id);
      types.emplace_back(h.h_mat[j], h.h_dx[j]);
      h.h_type[j] = id;
    } else {
      h.h_type[j] = it->second;
    }
  }
  const int T = (int)types.size();
  h.tt.n_types = T;
  const int G4 = 4 * G;
  Linv.assign((size_t)T * G * N * 16, 0.0);
  Cin.assign((size_t)T * G * N * 8, 0.0);
  Mp.assign((size_t)T * G4 * G4, 0.0);
  Kap.assign((size_t)T * G * G, 0.0);
  tdx.assign(T, 0.0);
  tsig.assign((size_t)T * G, 0.0);
  Lco.assign((size_t)T * G * N * 5, 0.0);
  std::vector<double> L(16), Li, KH((size_t)G4 * G4), IKH((size_t)G4 * G4), IKHinv;
  for (int t = 0; t < T; t++) {
    const int mt = types[t].first;
    const double dx = types[t].second;
    tdx[t] = dx;
    std::vector<double> H((size_t)G * 16, 0.0);
    for (int g = 0; g < G; g++) {
      const double sig = h.h_sigma_t[(size_t)mt * G + g];
      tsig[(size_t)t * G + g] = sig;
      const double al = dx / (h.h_v[g] * h.dt);
      for (int gp = 0; gp < G; gp++)
        Kap[((size_t)t * G + gp) * G + g] = dx / 4.0 * h.h_sigma_s[((size_t)mt * G + gp) * G + g];
      for (int m = 0; m < N; m++) {
        const double mu = h.h_mu[m];
        const double a = (fabs(mu) + dx * sig) / 2.0;
        const double Lm[16] = {a,   mu / 2.0, al / 2.0, 0.0,      -mu / 2.0, a,   0.0,       al / 2.0,
                               -al, 0.0,      al + a,   mu / 2.0, 0.0,       -al, -mu / 2.0, al + a};
        L.assign(Lm, Lm + 16);
        if (!invert(4, L, Li)) {
          set_error("a 4x4 angle block L_c is singular (zero width, cross section and speed term)");
          return OCI_E_SINGULAR;
        }
        const size_t o = ((size_t)t * G * N + (size_t)g * N + m);
        for (int k = 0; k < 16; k++) Linv[o * 16 + k] = Li[k];
        Lco[o * 5 + 0] = a;
        Lco[o * 5 + 1] = mu / 2.0;
        Lco[o * 5 + 2] = al / 2.0;
        Lco[o * 5 + 3] = al;
        Lco[o * 5 + 4] = al + a;
        // inflow enters rows 0,2 (mu > 0) or 1,3 (mu < 0) with factor |mu|
        const int ca = mu > 0 ? 0 : 1, cb = mu > 0 ? 2 : 3;
        for (int p = 0; p < 4; p++) {
          Cin[o * 8 + p * 2 + 0] = fabs(mu) * Li[p * 4 + ca];
          Cin[o * 8 + p * 2 + 1] = fabs(mu) * Li[p * 4 + cb];
        }
        for (int k = 0; k < 16; k++) H[(size_t)g * 16 + k] += h.h_w[m] * Li[k];
      }
    }
    // KH: block (g, gp) = Kap[gp->g] * H_gp ; IKH = I - KH ; Mp = IKH^{-1} K
    for (int g = 0; g < G; g++)
      for (int gp = 0; gp < G; gp++) {
        const double k = Kap[((size_t)t * G + gp) * G + g];
        for (int r = 0; r < 4; r++)
          for (int c = 0; c < 4; c++) KH[(size_t)(g * 4 + r) * G4 + gp * 4 + c] = k * H[(size_t)gp * 16 + r * 4 + c];
      }
    for (int r = 0; r < G4; r++)
      for (int c = 0; c < G4; c++) IKH[(size_t)r * G4 + c] = (r == c ? 1.0 : 0.0) - KH[(size_t)r * G4 + c];
    if (!invert(G4, IKH, IKHinv)) {
      set_error("the within-cell scalar-flux system (I - K H) is singular");
      return OCI_E_SINGULAR;
    }
    for (int r = 0; r < G4; r++)
      for (int gp = 0; gp < G; gp++)
        for (int c = 0; c < 4; c++) {
          // (IKHinv K)[r][(gp,c)] = sum_g IKHinv[r][(g,c)] * Kap[gp->g]
          double s = 0.0;
          for (int g = 0; g < G; g++) s += IKHinv[(size_t)r * G4 + g * 4 + c] * Kap[((size_t)t * G + gp) * G + g];
          Mp[(size_t)t * G4 * G4 + (size_t)r * G4 + gp * 4 + c] = s;
        }
  }
  return OCI_OK;
}

template <class T>
static int dev_upload(T **dst, const T *src, size_t n, cudaStream_t s) {
  CK(cudaMalloc(dst, n * sizeof(T) + 16));
  if (src) CK(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return OCI_OK;
}

static int build_graph(Handle &h, bool si, cudaGraphExec_t *out);

// ---------------------------------------------------------------- autotuner
// Launch shape of the sweep kernel (cells per block CB, angle chunks P per cell
// and group): every legal shape -- CB*G*P threads in [32, 256], P | N, shared
// memory <= 100 KB -- is timed over a few sweeps of this problem (CUDA events),
// and the fastest is kept for the graphs.  State is zeroed afterwards.
// OCI_AUTOTUNE=0 keeps the default shape.
// A candidate shape whose launch the runtime refuses (more blocks than can be
// co-resident for a cooperative launch, or an empty grid where not one block
// fits on an SM) is skipped by the autotuners rather than timed.
static bool launch_refused(cudaError_t e) {
  return e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorInvalidConfiguration ||
         e == cudaErrorLaunchOutOfResources;
}

static int autotune(Handle &h) {
  const char *at = hook_env("OCI_AUTOTUNE");
  if (at && at[0] == '0') return OCI_OK;
  const bool mx = h.precision == OCI_FP32_IR;
  if (h.solver == OCI_SOLVER_DENSE_LU || (h.precision != OCI_FP64 && !mx)) return OCI_OK;
  const size_t es = mx ? 4 : 8;
  struct Cand {
    int kind, cb, P;  // kind: kMxPlain (and the FP64 sweep), kMxTma, kMxReg
  };
  std::vector<Cand> cands;
  for (int cb : {32, 64, 128, 256})
    for (int P : {1, 2, 4, 8}) {
      if (h.N % P) continue;
      const int thr = cb * h.G * P;
      if (thr < 32 || thr > 256) continue;
      if (sweep_smem(h.N, h.G, cb, P, es) > 100 * 1024) continue;
      cands.push_back({kMxPlain, cb, P});
    }
  if (mx && h.tma_ok)
    for (int P : {1, 2, 4, 8})
      if (h.N % P == 0 && 64 * h.G * P <= 256 && mx_tma_smem(h, P) <= 200 * 1024) cands.push_back({kMxTma, 64, P});
  if (!mx && h.ordering != OCI_ORDER_RED_BLACK)  // FP64 register form
    for (int np : {2, 4, 8}) {
      if (h.N % np) continue;
      const int P = h.N / np;
      // blocks of 4 and 8 cells spread a small problem over more SMs (the FP64
      // pipe of one SM bounds a block's sweep); timed only where one launch
      // runs all sweeps of a step (below)
      for (int cb : {4, 8, 16, 32, 64}) {
        const int thr = cb * h.G * P;
        if (thr <= 256 && thr % 32 == 0 && thr >= (cb < 16 ? 32 : 64)) cands.push_back({kSweepReg64, cb, P});
      }
    }
  if (mx)
    for (int np : {2, 4, 8}) {
      if (h.N % np) continue;
      const int P = h.N / np;
      for (int cb : {16, 32, 64, 128}) {
        const int thr = cb * h.G * P;
        if (thr <= 256 && thr % 32 == 0 && thr >= 64) cands.push_back({kMxReg, cb, P});
        if (cb == 16 || cb == 128) {  // 16- and 128-cell tiles: persistent forms, 8 angles per thread
          if (np == 8 && thr <= 256 && thr % 32 == 0 && thr >= 64) cands.push_back({kMxTiledP, cb, P});
          continue;
        }
        if (thr <= 256 && cb <= 64) {
          cands.push_back({kMxTiled, cb, P});
          cands.push_back({kMxTiledP, cb, P});
          if (np <= 4 && cb >= 32 && thr % 32 == 0 &&
              mx_ms2_smem(h, cb, P, mx_tables_floats(h) * 4 <= 64 * 1024) <= 160 * 1024) {
            cands.push_back({kMxTiled2, cb, P});
            if (h.N == 16 && h.G == 1) cands.push_back({kMxTiled2Occ, cb, P});
          }
          if (np == 4 && cb == 32 && mx_w2_supported(h)) cands.push_back({kMxWarp2, 32, P});
          if (mx_tb_smem(h, cb, P, mx_tables_floats(h) * 4 <= 64 * 1024) <= 200 * 1024)
            cands.push_back({kMxTiledB, cb, P});
        }
      }
    }
  // OCI_MX_INNER=plain|tma|reg|tiled|tiledp|tiledb|two|twoocc|warp restricts the FP32 inner sweep to one kernel (for profiling)
  const char *only = hook_env("OCI_MX_INNER");
  if (mx && only) {  // a comma-separated list keeps several kernels (timed against one another)
    std::vector<int> want;
    std::string rest(only);
    while (!rest.empty()) {
      const size_t cut = rest.find(',');
      const std::string o = rest.substr(0, cut);
      rest = cut == std::string::npos ? "" : rest.substr(cut + 1);
      want.push_back(o == "tma"      ? kMxTma
                     : o == "reg"    ? kMxReg
                     : o == "tiled"  ? kMxTiled
                     : o == "tiledp" ? kMxTiledP
                     : o == "tiledb" ? kMxTiledB
                     : o == "two"    ? kMxTiled2
                     : o == "twoocc" ? kMxTiled2Occ
                     : o == "warp"   ? kMxWarp2
                                     : kMxPlain);
    }
    std::vector<Cand> keep;
    for (auto &c : cands)
      if (std::find(want.begin(), want.end(), c.kind) != want.end()) keep.push_back(c);
    if (!keep.empty()) cands.swap(keep);
  }
  // OCI_SWEEP_REG=0|1 restricts the FP64 Jacobi sweep to the staged / register form
  const char *sreg = hook_env("OCI_SWEEP_REG");
  if (!mx && sreg) {
    const int want = sreg[0] == '1' ? kSweepReg64 : kMxPlain;
    std::vector<Cand> keep;
    for (auto &c : cands)
      if (c.kind == want) keep.push_back(c);
    if (!keep.empty()) cands.swap(keep);
  }
  // OCI_SWEEP_SHAPE="cb,P" keeps one legal shape (the first of the remaining
  // candidates with that shape) without timing, so a profiler sees no tuning launches
  const char *shape = hook_env("OCI_SWEEP_SHAPE");
  if (shape) {
    int fcb = 0, fP = 0;
    if (sscanf(shape, "%d,%d", &fcb, &fP) == 2)
      for (auto &c : cands)
        if (c.cb == fcb && c.P == fP) {
          const Cand keep = c;
          cands.assign(1, keep);
          break;
        }
  }
  auto apply = [&](const Cand &c) {
    if (mx) {
      h.mx_kind = c.kind;
      h.mx_cb = c.cb;
      h.mx_P = c.P;
    } else {
      h.tune_cb = c.cb;
      h.tune_P = c.P;
      h.tune_reg = c.kind == kSweepReg64;
    }
  };
  if (cands.size() < 2) {
    if (cands.size() == 1) apply(cands[0]);
    return OCI_OK;
  }
  DevState &d = *h.h_ds;
  d.done = 0;
  d.fixed = 1;
  d.refine = 0;
  d.blk_i = 1;
  d.cur = 0;
  d.dcur = 0;
  d.max_iter = 0;        // no e history while timing
  d.k_max = 1 << 30;     // and no refinement decisions
  d.theta = 0.0;
  CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream));
  float best = 1e30f;
  Cand bc = cands[0];
  const int reps = 4;  // even: the two-sweep form runs two full passes
  for (auto &c : cands) {
    apply(c);
    // the persistent tiled FP32 sweep runs as one multi-sweep cooperative launch in
    // the graph: time it that way (reps sweeps in one launch)
    // (and so does the FP64 register form where all its blocks fit at once)
    const bool multi = (mx &&
                        (c.kind == kMxTiledP || c.kind == kMxTiled2 || c.kind == kMxTiled2Occ || c.kind == kMxWarp2) &&
                        h.mx_multi) ||
                       (!mx && c.kind == kSweepReg64 && (sweep_cl_grid(h) > 0 || sweep_ms_grid(h) > 0));
    auto sweep = [&]() {
      if (mx) launch_mx_inner(h, cudaGraphConditionalHandle{}, 0);
      else launch_oci_sweep(h, cudaGraphConditionalHandle{}, 0);
    };
    if (!mx && c.kind == kSweepReg64 && c.cb < 16 && !multi) continue;
    h.mx_tune_sweeps = multi ? 1 : 0;
    sweep();
    float ms = 1e30f;
    for (int t = 0; t < 2; t++) {  // the faster of two timings: one disturbed launch picks no shape
      CK(cudaEventRecord(h.ev0, h.stream));
      if (multi) {
        h.mx_tune_sweeps = reps;
        sweep();
      } else {
        for (int r = 0; r < reps; r++) sweep();
      }
      CK(cudaEventRecord(h.ev1, h.stream));
      CK(cudaEventSynchronize(h.ev1));
      const cudaError_t le = cudaGetLastError();
      if (launch_refused(le)) {
        ms = 1e30f;
        break;
      }
      if (le != cudaSuccess) return cuda_fail(le, "timing a sweep shape");
      float m = 0.f;
      cudaEventElapsedTime(&m, h.ev0, h.ev1);
      ms = std::min(ms, m);
    }
    h.mx_tune_sweeps = 0;
    if (ms < best) {
      best = ms;
      bc = c;
    }
  }
  if (best >= 1e30f) return set_error("no sweep shape could be launched on this device"), OCI_E_CUDA;
  apply(bc);
  h.tune_us = 1e3 * best / reps;
  const size_t nPsi = (size_t)h.G * h.N * 4 * h.Jp;
  CK(cudaMemsetAsync(h.Psi[0], 0, nPsi * 8, h.stream));
  CK(cudaMemsetAsync(h.Psi[1], 0, nPsi * 8, h.stream));
  if (mx) {
    const size_t nPsi32 = (size_t)h.G * h.N * 4 * std::max<size_t>(h.Jp, (h.J + 127) / 128 * 128);
    CK(cudaMemsetAsync(h.delta[0], 0, nPsi32 * 4, h.stream));
    CK(cudaMemsetAsync(h.delta[1], 0, nPsi32 * 4, h.stream));
  }
  std::memset(h.h_ds, 0, sizeof(DevState));
  h.h_ds->done = 1;
  h.h_ds->spin = kGridSpin;
  CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  return OCI_OK;
}

// FP64 red-black sweep on ping-pong buffers: the staged and the register form
// over the legal shapes, each timed (CUDA events) as a few sweeps of two half
// sweeps, on the first switch to red-black order.  The timing keeps the state:
// with the device state marked in place, every timed sweep reads Psi[cur] and
// writes only Psi[cur^1], and the state record is restored afterwards.
// OCI_RB_SHAPE="s,cb,P" or "r,cb,P" keeps one staged / register shape without
// timing; OCI_AUTOTUNE=0 or OCI_SWEEP_SHAPE leave the Jacobi staged shape in use.
static int tune_rb64(Handle &h) {
  if (h.precision != OCI_FP64 || h.solver == OCI_SOLVER_DENSE_LU || !h.rb_pingpong) return OCI_OK;
  struct RbC {
    bool reg;
    int cb, P;
  };
  std::vector<RbC> rcs;
  for (int cb : {32, 64, 128, 256})
    for (int P : {1, 2, 4, 8}) {
      const int thr = cb * h.G * P;
      if (h.N % P || thr < 32 || thr > 256 || sweep_smem(h.N, h.G, cb, P, 8) > 100 * 1024) continue;
      rcs.push_back({false, cb, P});
    }
  for (int np : {2, 4, 8}) {
    if (h.N % np) continue;
    const int P = h.N / np;
    for (int cb : {16, 32, 64}) {
      const int thr = cb * h.G * P;
      if (thr <= 256 && thr % 32 == 0 && thr >= 64) rcs.push_back({true, cb, P});
    }
  }
  auto apply = [&](const RbC &c) {
    h.rb_reg = c.reg;
    h.rb_cb = c.cb;
    h.rb_P = c.P;
  };
  const char *force = hook_env("OCI_RB_SHAPE");
  if (force) {
    char k = 0;
    int fcb = 0, fP = 0;
    if (sscanf(force, "%c,%d,%d", &k, &fcb, &fP) == 3)
      for (auto &c : rcs)
        if (c.reg == (k == 'r') && c.cb == fcb && c.P == fP) {
          apply(c);
          return OCI_OK;
        }
    return set_error("OCI_RB_SHAPE names no legal red-black shape for this N, G"), OCI_E_INVAL;
  }
  const char *at = hook_env("OCI_AUTOTUNE");
  if ((at && at[0] == '0') || hook_env("OCI_SWEEP_SHAPE") || rcs.size() < 2) return OCI_OK;
  // the handle's ordering, red-black shape and state record are put back on
  // every path, so a failed timing leaves the handle as it was
  const DevState saved = *h.h_ds;
  const int ordering = h.ordering;
  const RbC before{h.rb_reg, h.rb_cb, h.rb_P};
  const int reps = 4;
  float best = 1e30f;
  RbC bc = rcs[0];
  auto time_all = [&]() -> int {
    DevState &d = *h.h_ds;
    d.done = 0;
    d.fixed = 1;
    d.max_iter = 0;  // no e history while timing
    d.inplace = 1;   // no flip of cur: Psi[cur] is only read
    CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream));
    h.ordering = OCI_ORDER_RED_BLACK;
    for (auto &c : rcs) {
      apply(c);
      launch_oci_sweep(h, cudaGraphConditionalHandle{}, 0);
      float ms = 1e30f;
      for (int t = 0; t < 2; t++) {  // the faster of two timings
        CK(cudaEventRecord(h.ev0, h.stream));
        for (int r = 0; r < reps; r++) launch_oci_sweep(h, cudaGraphConditionalHandle{}, 0);
        CK(cudaEventRecord(h.ev1, h.stream));
        CK(cudaEventSynchronize(h.ev1));
        CK(cudaGetLastError());
        float m = 0.f;
        cudaEventElapsedTime(&m, h.ev0, h.ev1);
        ms = std::min(ms, m);
      }
      if (ms < best) {
        best = ms;
        bc = c;
      }
    }
    return OCI_OK;
  };
  const int rc = time_all();
  h.ordering = ordering;
  apply(rc ? before : bc);
  if (!rc) h.rb_tune_us = 1e3 * best / reps;
  *h.h_ds = saved;
  cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream);
  const cudaError_t e = cudaStreamSynchronize(h.stream);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "restoring the state after red-black timing");
  return OCI_OK;
}

// Red-black FP32 inner sweep of the mixed form: kernels (one sweep per pass,
// kMxRB; two sweeps per pass, kMxRB2) and shapes (tile T cells, P angle
// chunks), each timed as one launch of four sweeps (as the graph runs them);
// the Jacobi choice is kept for a switch back.  The handle's state is saved
// and restored around the timing.  OCI_MX_RB=1|2 keeps one kernel.
static int tune_rb(Handle &h) {
  h.mx_jac_kind = h.mx_kind;
  h.mx_jac_cb = h.mx_cb;
  h.mx_jac_P = h.mx_P;
  struct RbCand {
    int kind, T, P;
  };
  std::vector<RbCand> cands;
  const char *only = hook_env("OCI_MX_RB");
  const bool stage = mx_tables_floats(h) * 4 <= 64 * 1024;
  for (int T : {32, 64})
    for (int np : {2, 4, 8}) {
      if (h.N % np) continue;
      const int P = h.N / np, thr = (T / 2) * h.G * P;
      if (thr > 256 || thr % 32) continue;
      if (!(only && only[0] == '2')) cands.push_back({kMxRB, T, P});
      if (!(only && only[0] == '1') && np <= 4 && mx_rb2_smem(h, T, P, stage) <= 160 * 1024)
        cands.push_back({kMxRB2, T, P});
    }
  if (cands.empty()) return set_error("no red-black inner-sweep shape fits this N, G"), OCI_E_INVAL;
  const char *shape = hook_env("OCI_SWEEP_SHAPE");
  if (shape) {
    int fT = 0, fP = 0;
    if (sscanf(shape, "%d,%d", &fT, &fP) == 2)
      for (auto &c : cands)
        if (c.T == fT && c.P == fP) {
          const RbCand keep = c;
          cands.assign(1, keep);
          break;
        }
  }
  auto apply = [&](const RbCand &c) {
    h.mx_kind = c.kind;
    h.mx_cb = c.T;
    h.mx_P = c.P;
  };
  if (cands.size() == 1) {
    apply(cands[0]);
    return OCI_OK;
  }
  // the inner-sweep choice and the state record are put back on a failure
  const DevState saved = *h.h_ds;
  const RbCand before{h.mx_kind, h.mx_cb, h.mx_P};
  float best = 1e30f;
  RbCand bc = cands[0];
  const int reps = 4;
  auto time_all = [&]() -> int {
    DevState d = saved;
    d.done = 0;
    d.fixed = 1;
    d.refine = 0;
    d.blk_i = 1;
    d.dcur = 0;
    d.max_iter = 0;
    d.k_max = 1 << 30;
    d.theta = 0.0;
    d.spin = kGridSpin;
    for (auto &c : cands) {
      apply(c);
      d.inplace = c.kind == kMxRB;
      *h.h_ds = d;
      CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream));
      h.mx_tune_sweeps = 1;
      launch_mx_inner(h, cudaGraphConditionalHandle{}, 0);
      float ms = 1e30f;
      for (int t = 0; t < 2; t++) {  // the faster of two timings: one disturbed launch picks no shape
        CK(cudaEventRecord(h.ev0, h.stream));
        h.mx_tune_sweeps = reps;
        launch_mx_inner(h, cudaGraphConditionalHandle{}, 0);
        CK(cudaEventRecord(h.ev1, h.stream));
        CK(cudaEventSynchronize(h.ev1));
        const cudaError_t le = cudaGetLastError();
        if (launch_refused(le)) {
          ms = 1e30f;
          break;
        }
        if (le != cudaSuccess) return cuda_fail(le, "timing a red-black inner sweep");
        float m = 0.f;
        cudaEventElapsedTime(&m, h.ev0, h.ev1);
        ms = std::min(ms, m);
      }
      h.mx_tune_sweeps = 0;
      if (ms < best) {
        best = ms;
        bc = c;
      }
    }
    if (best >= 1e30f) return set_error("no red-black inner sweep could be launched on this device"), OCI_E_CUDA;
    return OCI_OK;
  };
  const int rc = time_all();
  h.mx_tune_sweeps = 0;
  apply(rc ? before : bc);
  if (!rc) h.tune_us = 1e3 * best / reps;
  *h.h_ds = saved;
  cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream);
  const cudaError_t e = cudaStreamSynchronize(h.stream);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "restoring the state after red-black timing");
  return OCI_OK;
}

void free_batch(Batch *b);

static void free_handle(Handle *h) {
  if (!h) return;
  if (h->batch) {
    free_batch(h->batch);
    h->batch = nullptr;
  }
  if (h->stream) cudaStreamSynchronize(h->stream);
  gmres_free(*h);
  void *ptrs[] = {h->Psi[0], h->Psi[1], h->tc,        h->psi_prev,  h->phi,          h->phi_si[0], h->phi_si[1],
                  h->Q,      h->inc,    h->type,      h->mu,        h->w,            h->v,         h->tt.Linv,
                  h->tt.Cin, h->tt.Mp,  h->tt.Kap,    h->tt.dx,     h->tt.sig,       h->si_z,      h->si_uin,
                  h->LU,     h->piv,    h->partials,  h->bal_partials, h->bal,       h->e_hist,    h->ds,
                  h->stage,  h->delta[0], h->delta[1], h->z32, h->w32, h->tt.Lco, h->tt.Linv32, h->tt.Cin32,
                  h->tt.Mp32, h->tc_img, h->tc_items, h->si_maps, h->si_segin, h->counter, h->psi_user, h->gbar, h->mu32,
                  h->yc,     h->tt.Win, h->tc_img_h, h->tc_z};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (h->h_ds) cudaFreeHost(h->h_ds);
  if (h->h_bal) cudaFreeHost(h->h_bal);
  if (h->g_oci) cudaGraphExecDestroy(h->g_oci);
  if (h->g_si) cudaGraphExecDestroy(h->g_si);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete static_cast<oci_handle *>(h);
}

static int setup_impl(const oci_problem *p, oci_handle *h) {
  h->J = p->J;
  h->N = p->N;
  h->G = p->G;
  h->n_mat = p->n_mat;
  h->Jp = (p->J + 31) / 32 * 32;
  h->dt = p->dt;
  h->tol = p->tol;
  h->max_iter = p->max_iter;
  h->precision = p->precision;
  h->guess = p->guess;
  h->solver = p->solver == OCI_SOLVER_AUTO ? OCI_SOLVER_STRUCTURED : p->solver;
  h->stream = (cudaStream_t)p->stream;
  {
    const char *ng = hook_env("OCI_NO_GRAPH");
    h->no_graph = ng && ng[0] == '1';
  }
  CK(cudaGetDevice(&h->device));
  const size_t J = h->J, N = h->N, G = h->G, Jp = h->Jp;
  h->h_dx.assign(p->dx, p->dx + J);
  h->h_mat.assign(p->mat, p->mat + J);
  h->h_sigma_t.assign(p->sigma_t, p->sigma_t + (size_t)p->n_mat * G);
  h->h_sigma_s.assign(p->sigma_s, p->sigma_s + (size_t)p->n_mat * G * G);
  h->h_v.assign(p->v, p->v + G);
  gauss_legendre(h->N, h->h_mu, h->h_w);

  std::vector<double> Linv, Cin, Mp, Kap, tdx, tsig, Lco;
  int rc = build_tables(*h, Linv, Cin, Mp, Kap, tdx, tsig, Lco);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  const size_t nPsi = G * N * 4 * Jp;
  CK(cudaMalloc(&h->Psi[0], nPsi * 8));
  CK(cudaMalloc(&h->Psi[1], nPsi * 8));
  CK(cudaMalloc(&h->tc, nPsi * 8));
  CK(cudaMalloc(&h->yc, G * 4 * Jp * 8));
  CK(cudaMalloc(&h->psi_prev, G * N * 2 * Jp * 8));
  CK(cudaMalloc(&h->phi, G * 4 * Jp * 8));
  CK(cudaMalloc(&h->stage, nPsi * 8));
  if (h->guess == OCI_GUESS_USER) {
    CK(cudaMalloc(&h->psi_user, nPsi * 8));
    CK(cudaMemsetAsync(h->psi_user, 0, nPsi * 8, s));
  }
  CK(cudaMemsetAsync(h->Psi[0], 0, nPsi * 8, s));
  CK(cudaMemsetAsync(h->Psi[1], 0, nPsi * 8, s));
  CK(cudaMemsetAsync(h->tc, 0, nPsi * 8, s));
  CK(cudaMemsetAsync(h->yc, 0, G * 4 * Jp * 8, s));
  CK(cudaMemsetAsync(h->psi_prev, 0, G * N * 2 * Jp * 8, s));
  CK(cudaMemsetAsync(h->phi, 0, G * 4 * Jp * 8, s));
  std::vector<int32_t> typ(Jp, 0);
  for (size_t j = 0; j < J; j++) typ[j] = h->h_type[j];
  if ((rc = dev_upload(&h->type, typ.data(), Jp, s))) return rc;
  if ((rc = dev_upload(&h->mu, h->h_mu.data(), N, s))) return rc;
  if ((rc = dev_upload(&h->w, h->h_w.data(), N, s))) return rc;
  if ((rc = dev_upload(&h->v, h->h_v.data(), G, s))) return rc;
  if ((rc = dev_upload(&h->tt.Linv, Linv.data(), Linv.size(), s))) return rc;
  if ((rc = dev_upload(&h->tt.Cin, Cin.data(), Cin.size(), s))) return rc;
  {
    std::vector<double> Win(Cin.size());
    for (size_t o = 0; o < Cin.size() / 8; o++)
      for (int k = 0; k < 8; k++) Win[o * 8 + k] = h->h_w[o % N] * Cin[o * 8 + k];
    if ((rc = dev_upload(&h->tt.Win, Win.data(), Win.size(), s))) return rc;
    CK(cudaStreamSynchronize(s));  // Win is a local vector
  }
  if ((rc = dev_upload(&h->tt.Mp, Mp.data(), Mp.size(), s))) return rc;
  if ((rc = dev_upload(&h->tt.Kap, Kap.data(), Kap.size(), s))) return rc;
  if ((rc = dev_upload(&h->tt.dx, tdx.data(), tdx.size(), s))) return rc;
  if ((rc = dev_upload(&h->tt.sig, tsig.data(), tsig.size(), s))) return rc;
  std::vector<double> inc(2 * G * N * 2, 0.0);
  if (p->inc_left) std::memcpy(inc.data(), p->inc_left, G * N * 2 * 8);
  if (p->inc_right) std::memcpy(inc.data() + G * N * 2, p->inc_right, G * N * 2 * 8);
  if ((rc = dev_upload(&h->inc, inc.data(), inc.size(), s))) return rc;
  if (p->Q) {
    if ((rc = dev_upload(&h->Q, (const double *)nullptr, G * 4 * Jp, s))) return rc;
    CK(cudaMemcpyAsync(h->stage, p->Q, J * G * 4 * 8, cudaMemcpyHostToDevice, s));
    launch_transpose_in(*h, h->stage, h->Q, (int)(G * 4));
  }
  if (p->psi_init) {
    CK(cudaMemcpyAsync(h->stage, p->psi_init, J * G * N * 2 * 8, cudaMemcpyHostToDevice, s));
    launch_transpose_in(*h, h->stage, h->psi_prev, (int)(G * N * 2));
  }
  // reduction scratch
  SweepCfg sc = sweep_config(*h);
  int np = sc.grid;
  np = std::max(np, si_partials(*h));
  np = std::max(np, dense_partials(*h));
  np = std::max(np, mx_partials(*h));
  np = std::max(np, tc_partials(*h));
  np = std::max(np, h->J + 64);  // any sweep shape down to one cell per block
  h->n_partials = np;
  CK(cudaMalloc(&h->partials, (size_t)np * 8));
  CK(cudaMalloc(&h->counter, sizeof(unsigned)));
  CK(cudaMemsetAsync(h->counter, 0, sizeof(unsigned), s));
  CK(cudaMalloc(&h->gbar, 2 * sizeof(unsigned)));
  CK(cudaMemsetAsync(h->gbar, 0, 2 * sizeof(unsigned), s));
  {
    const char *mm = hook_env("OCI_MX_MULTI");  // 0: one inner sweep per launch in the graph as well
    h->mx_multi = !(mm && mm[0] == '0');
    const char *rf = hook_env("OCI_RB_FP64");  // "inplace": FP64 red-black half sweeps update Psi[cur] in place
    h->rb_pingpong = !(rf && rf[0] == 'i');
    const char *cv = hook_env("OCI_MX_OUTER_CVT");  // "hw": compiler conversions in the FP64 refinement
    h->mx_hwcvt = (cv && cv[0] == 'h') ? 1 : 0;
  }
  const int nblk_carry = (h->J + 31) / 32;
  CK(cudaMalloc(&h->bal_partials, (size_t)nblk_carry * G * 8 * 8));
  CK(cudaMalloc(&h->bal, G * 10 * 8));
  CK(cudaMemsetAsync(h->bal, 0, G * 10 * 8, s));
  h->e_hist_cap = h->max_iter;
  CK(cudaMalloc(&h->e_hist, (size_t)h->e_hist_cap * 8));
  CK(cudaMalloc(&h->ds, sizeof(DevState)));
  CK(cudaMallocHost(&h->h_ds, sizeof(DevState)));
  CK(cudaMallocHost(&h->h_bal, G * 10 * 8));
  std::memset(h->h_ds, 0, sizeof(DevState));
  h->h_ds->done = 1;
  h->h_ds->spin = kGridSpin;
  CK(cudaMemcpyAsync(h->ds, h->h_ds, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(cudaEventCreate(&h->ev0));
  CK(cudaEventCreate(&h->ev1));
  if (h->solver == OCI_SOLVER_DENSE_LU) {
    if ((rc = dense_setup(*h))) return rc;
  }
  CK(cudaFuncSetAttribute(k_oci_sweep_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CK(cudaFuncSetAttribute(k_oci_sweep_rb_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CK(cudaFuncSetAttribute(k_oci_sweep_rbpp_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  if (h->precision != OCI_FP64) {
    auto to32 = [](const std::vector<double> &a) {
      std::vector<float> f(a.size());
      for (size_t i = 0; i < a.size(); i++) f[i] = (float)a[i];
      return f;
    };
    std::vector<float> L32 = to32(Linv), C32 = to32(Cin), M32 = to32(Mp), W32 = to32(h->h_w);
    if ((rc = dev_upload(&h->tt.Lco, Lco.data(), Lco.size(), s))) return rc;
    if ((rc = dev_upload(&h->tt.Linv32, L32.data(), L32.size(), s))) return rc;
    if ((rc = dev_upload(&h->tt.Cin32, C32.data(), C32.size(), s))) return rc;
    if ((rc = dev_upload(&h->tt.Mp32, M32.data(), M32.size(), s))) return rc;
    if ((rc = dev_upload(&h->w32, W32.data(), W32.size(), s))) return rc;
    const std::vector<float> MU32 = to32(h->h_mu);
    if ((rc = dev_upload(&h->mu32, MU32.data(), MU32.size(), s))) return rc;
    CK(cudaStreamSynchronize(s));  // host vectors of the uploads go out of scope
    // FP32 correction arrays: room for both layouts ([R][Jp], and tile-major
    // with tiles of up to 128 cells)
    const size_t nPsi32 = (size_t)G * N * 4 * std::max<size_t>(Jp, (h->J + 127) / 128 * 128);
    CK(cudaMalloc(&h->delta[0], nPsi32 * 4));
    CK(cudaMalloc(&h->delta[1], nPsi32 * 4));
    CK(cudaMalloc(&h->z32, nPsi32 * 4));
    CK(cudaMemsetAsync(h->delta[0], 0, nPsi32 * 4, s));
    CK(cudaMemsetAsync(h->delta[1], 0, nPsi32 * 4, s));
    CK(cudaMemsetAsync(h->z32, 0, nPsi32 * 4, s));
    if ((rc = mx_set_attributes())) return rc;
    if (h->precision == OCI_FP32_IR && (rc = mx_tma_setup(*h))) return rc;
    if (h->precision == OCI_TF32_IR) {
      h->mx_theta = 2e-2;
      h->mx_kmax = 24;
    } else if (h->precision == OCI_BF16X3_IR) {
      h->mx_theta = 2e-3;
      h->mx_kmax = 48;
    }
    if (h->precision == OCI_TF32_IR || h->precision == OCI_BF16X3_IR) {
      // The streamed kernel takes a tile of 128 cells once per cell type in it; the
      // resident-inverse kernels (behind a test hook) need one type per tile.  Passes
      // are bounded at twice the tiles, so that many small regions do not multiply the
      // work, and the per-type inverses at 2^28 entries.
      const bool streamed = tc_big_used(*h);
      size_t passes = 0;
      const size_t ntiles = (size_t)(h->J + 127) / 128;
      for (int j0 = 0; j0 < h->J; j0 += 128) {
        std::vector<int32_t> seen;
        for (int j = j0; j < std::min(h->J, j0 + 128); j++)
          if (std::find(seen.begin(), seen.end(), h->h_type[j]) == seen.end()) seen.push_back(h->h_type[j]);
        passes += seen.size();
        if (!streamed && seen.size() > 1) {
          set_error("the resident-inverse tensor-core kernels need one cell type per aligned tile of 128 cells");
          return OCI_E_INVAL;
        }
      }
      if (passes > 2 * ntiles) {
        set_error("the tensor-core forms take a 128-cell tile once per cell type in it; these cell types "
                  "would need more than twice the tiles");
        return OCI_E_INVAL;
      }
      // dense A = L_c - S per type (Eqs. Aj, scatter, fullOCIlhs) and its inverse
      const int n = 4 * h->N * h->G, T = h->tt.n_types;
      if ((size_t)T * n * n > ((size_t)1 << 28)) {
        set_error("the tensor-core forms keep one dense inverse per cell type: too many types for this cell size");
        return OCI_E_INVAL;
      }
      std::vector<double> Ainv_all((size_t)T * n * n), A((size_t)n * n), Ai;
      for (int t = 0; t < T; t++) {
        std::fill(A.begin(), A.end(), 0.0);
        for (int g = 0; g < h->G; g++)
          for (int m = 0; m < h->N; m++) {
            const double *Lc = &Lco[(((size_t)t * h->G + g) * h->N + m) * 5];
            const double a = Lc[0], hm = Lc[1], ha = Lc[2], al = Lc[3], aa = Lc[4];
            const double L[16] = {a, hm, ha, 0.0, -hm, a, 0.0, ha, -al, 0.0, aa, hm, 0.0, -al, -hm, aa};
            const int r0 = (g * h->N + m) * 4;
            for (int r = 0; r < 4; r++)
              for (int c = 0; c < 4; c++) A[(size_t)(r0 + r) * n + r0 + c] += L[r * 4 + c];
          }
        for (int g = 0; g < h->G; g++)
          for (int gp = 0; gp < h->G; gp++) {
            const double k = Kap[((size_t)t * h->G + gp) * h->G + g];
            for (int m = 0; m < h->N; m++)
              for (int nn = 0; nn < h->N; nn++)
                for (int q = 0; q < 4; q++)
                  A[(size_t)((g * h->N + m) * 4 + q) * n + (gp * h->N + nn) * 4 + q] -= k * h->h_w[nn];
          }
        if (!invert(n, A, Ai)) return set_error("a cell matrix A_j is singular"), OCI_E_SINGULAR;
        std::copy(Ai.begin(), Ai.end(), Ainv_all.begin() + (size_t)t * n * n);
      }
      if ((rc = tc_build_images(*h, Ainv_all))) return rc;
      if ((rc = tc_prepare(*h))) return rc;
    }
    const char *km = hook_env("OCI_MX_KMAX");
    if (km) h->mx_kmax = std::max(1, atoi(km));
    const char *th = hook_env("OCI_MX_THETA");
    if (th) h->mx_theta = atof(th);
  }
  if ((rc = autotune(*h))) return rc;
  if ((rc = build_graph(*h, false, &h->g_oci))) return rc;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return OCI_OK;
}

// Body of one iteration of the convergence loop (sweep + finalize).
// Inner sweep of a mixed form with its norm, stop rule and refinement decision.
static void launch_mx_sweep(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  if (h.precision == OCI_FP32_IR) {
    launch_mx_inner(h, cond, use_cond);  // norm and stop rule fused in
  } else if (tc_big_used(h)) {
    launch_tc_big(h, cond, use_cond);  // 4NG > 128: M-tiled, A^{-1} streamed per K-chunk
  } else if (tc_pipe_ok(h)) {
    launch_tc_pipe(h, cond, use_cond);  // persistent pipelined tensor-core sweep, norm fused in
  } else {
    launch_tc_inner(h);
    launch_mx_finalize(h, cond, use_cond);
  }
}

static void launch_body(Handle &h, bool si, cudaGraphConditionalHandle cond, int use_cond) {
  if (si) {
    launch_si_sweep(h);
    launch_finalize(h, h.partials, si_partials(h), cond, use_cond);
  } else if (h.precision != OCI_FP64) {
    launch_mx_sweep(h, cond, use_cond);
    launch_mx_outer(h, 1);
  } else if (h.solver == OCI_SOLVER_DENSE_LU) {
    launch_dense_sweep(h);
    launch_finalize(h, h.partials, dense_partials(h), cond, use_cond);
  } else {
    launch_oci_sweep(h, cond, use_cond);  // norm and stop rule fused in
  }
}

static int build_graph(Handle &h, bool si, cudaGraphExec_t *out) {
  cudaGraph_t graph;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  CK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = h.stream;
  h.stream = cs;
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  const bool mx = !si && h.precision != OCI_FP64;
  if (e == cudaSuccess && !mx) {
    launch_body(h, si, cond, 1);
    e = cudaStreamEndCapture(cs, &body);
  } else if (e == cudaSuccess) {
    // mixed forms: the FP64 refinement sits under an IF node whose value the
    // sweep's stop-rule block sets, so a sweep without refinement launches
    // nothing after the inner kernel
    launch_mx_sweep(h, cond, 1);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle cref{};
    cudaGraphNodeParams ip = {};
    cudaGraphNode_t ifn;
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cref, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = cref;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      e = cudaGraphAddNode(&ifn, cg, deps, nullptr, nd, &ip);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies);
    cudaError_t e2 = cudaStreamEndCapture(cs, &body);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) {
      cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        launch_mx_outer(h, 1);
        e = cudaStreamEndCapture(cs, &ifbody);
      }
    }
    if (e == cudaSuccess) h.mx_cond_ref = (unsigned long long)cref;
  }
  h.stream = saved;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    // A capture that failed inside a conditional node's body leaves the parent
    // graph in a state that the driver does not survive destroying (a failed
    // kernel launch there crashed the process in cudaGraphDestroy): the graph
    // is left to the process's exit and the error is returned.
    return cuda_fail(e, "capturing the convergence loop");
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return OCI_OK;
}

// ---------------------------------------------------------------- stepping
// Spin limit of the cooperative kernels' grid barrier for the coming step:
// kGridSpin, or the test hook OCI_TEST_SPIN_LIMIT (an integer >= 0; 0 makes
// every block that is not the last to arrive give up at once, so the step ends
// with OCI_E_TIMEOUT without any wait).
static long long step_spin_limit() {
  const char *v = hook_env("OCI_TEST_SPIN_LIMIT");
  if (!v) return kGridSpin;
  char *end = nullptr;
  const long long x = strtoll(v, &end, 10);
  return (end != v && x >= 0 && x <= kGridSpin) ? x : kGridSpin;
}

static int begin_iteration(Handle &h, int fixed, int cap) {
  DevState &d = *h.h_ds;
  d.spin = step_spin_limit();
  d.l = 0;
  d.status = OCI_OK;
  d.done = 0;
  d.max_iter = cap;
  d.fixed = fixed;
  d.tol = h.tol;
  d.e = d.e_prev = d.rho = 0.0;
  d.dcur = 0;
  d.blk_i = 0;
  d.refine = 0;
  d.applied = 0;
  d.k_max = h.mx_kmax;
  d.n_refine = 0;
  d.theta = h.mx_theta;
  d.e_blk0 = 0.0;
  d.inplace = (h.ordering == OCI_ORDER_RED_BLACK && h.precision == OCI_FP64 && h.solver != OCI_SOLVER_DENSE_LU &&
               !h.rb_pingpong) ||
              h.mx_kind == kMxRB;
  d.cond_ref = h.mx_cond_ref;  // read only by kernels launched from the graph (use_cond)
  CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream));
  if (h.gbar) CK(cudaMemsetAsync(h.gbar, 0, 2 * sizeof(unsigned), h.stream));  // grid barrier count
  return OCI_OK;
}

static int run_step(Handle &h, bool si, oci_stats *st) {
  if (h.part_pending) return set_error("a sweep split by oci_iterate_part is not finished"), OCI_E_STATE;
  h.tc_fresh = 0;
  const size_t nPsi = (size_t)h.G * h.N * 4 * h.Jp;
  cudaStream_t s = h.stream;
  if (h.guess == OCI_GUESS_ZERO) CK(cudaMemsetAsync(h.Psi[h.h_ds->cur], 0, nPsi * 8, s));
  if (h.guess == OCI_GUESS_USER)
    CK(cudaMemcpyAsync(h.Psi[h.h_ds->cur], h.psi_user, nPsi * 8, cudaMemcpyDeviceToDevice, s));
  int rc = begin_iteration(h, 0, h.max_iter);
  if (rc) return rc;
  if (si) {
    launch_si_phi_from_psi(h, nullptr);
  } else if (h.precision != OCI_FP64) {
    launch_dense_step_const(h);  // c (not pre-multiplied)
    launch_mx_outer(h, 0);       // FP64 residual of the initial iterate
  } else if (h.solver == OCI_SOLVER_DENSE_LU) {
    launch_dense_step_const(h);
  } else {
    launch_step_const(h);
  }
  cudaGraphExec_t g = si ? h.g_si : h.g_oci;
  CK(cudaEventRecord(h.ev0, s));
  if (!si && h.accel == OCI_ACCEL_GMRES) {
    // Krylov acceleration: GMRES on (I - T) x = b, one sweep per Krylov vector
    int sweeps = 0, status = OCI_E_NOCONV;
    double e = 0.0;
    rc = gmres_solve(h, h.tol * h.gm_factor, h.max_iter, sweeps, e, status);
    if (rc) return rc;
    DevState &d = *h.h_ds;
    d.l = sweeps;
    d.e = e;
    d.rho = 0.0;
    d.status = status;
    d.done = 1;
    CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, s));
  } else if (h.no_graph) {
    // host-driven loop over the same kernels (for profilers that do not
    // descend into conditional graph bodies): batches of sweeps, each kernel
    // returns at once when the device state says the step is done
    cudaGraphConditionalHandle none{};
    for (int done_sweeps = 0; done_sweeps < h.max_iter;) {
      const int batch = std::min(16, h.max_iter - done_sweeps);
      for (int i = 0; i < batch; i++) launch_body(h, si, none, 0);
      done_sweeps += batch;
      CK(cudaMemcpyAsync(h.h_ds, h.ds, sizeof(DevState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h.h_ds->done) break;
    }
  } else {
    CK(cudaGraphLaunch(g, s));
  }
  CK(cudaEventRecord(h.ev1, s));
  if (!si && h.precision != OCI_FP64) launch_mx_settle(h, 0);
  launch_carry(h);  // device-guarded: commits only a converged step
  CK(cudaMemcpyAsync(h.h_ds, h.ds, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h.h_bal, h.bal, (size_t)h.G * 10 * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h.ev0, h.ev1);
  const DevState &d = *h.h_ds;
  h.last_iters = d.l;
  if (d.status == OCI_OK) h.t += h.dt;
  if (st) {
    st->iters = d.l;
    st->status = d.status;
    st->e_last = d.e;
    st->rho_e_last = d.rho;
    st->t = h.t;
    st->seconds = ms * 1e-3;
    st->refinements = (si || h.precision == OCI_FP64) ? 0 : d.n_refine;
    st->reserved = 0;
    st->balance_rel[0] = st->balance_rel[1] = 0.0;
    if (d.status == OCI_OK) {
      for (int g = 0; g < h.G; g++)
        for (int b = 0; b < 2; b++) {
          const double *x = h.h_bal + g * 10 + b * 5;
          const double r = x[0] + x[1] + x[2] - x[3] - x[4];
          const double sc = fabs(x[0]) + fabs(x[1]) + fabs(x[2]) + fabs(x[3]) + fabs(x[4]);
          const double rel = sc > 0 ? fabs(r) / sc : 0.0;
          if (rel > st->balance_rel[b]) st->balance_rel[b] = rel;
        }
    }
  }
  if (d.status == OCI_E_NOCONV) {
    char buf[160];
    snprintf(buf, sizeof buf, "no convergence after %d sweeps (e = %.3e)", d.l, d.e);
    set_error(buf);
  } else if (d.status == OCI_E_NONFINITE) {
    set_error("the convergence norm is not finite");
  } else if (d.status == OCI_E_TIMEOUT) {
    set_error("a bounded device-side wait gave up (step not committed)");
  }
  return d.status;
}

static int run_fixed(Handle &h, bool si, int n, double *e_hist) {
  if (n < 0) return set_error("n must be >= 0"), OCI_E_INVAL;
  if (h.part_pending) return set_error("a sweep split by oci_iterate_part is not finished"), OCI_E_STATE;
  h.tc_fresh = 0;
  if (n > h.e_hist_cap) {
    cudaFree(h.e_hist);
    h.e_hist_cap = n;
    CK(cudaMalloc(&h.e_hist, (size_t)n * 8));
  }
  int rc = begin_iteration(h, 1, h.e_hist_cap);
  if (rc) return rc;
  const bool mx = !si && h.precision != OCI_FP64;
  if (si) {
    launch_si_phi_from_psi(h, nullptr);
  } else if (mx) {
    launch_dense_step_const(h);
    launch_mx_outer(h, 0);
  } else if (h.solver == OCI_SOLVER_DENSE_LU) {
    launch_dense_step_const(h);
  } else {
    launch_step_const(h);
  }
  cudaGraphConditionalHandle none{};
  for (int i = 0; i < n; i++) launch_body(h, si, none, 0);
  if (mx) {
    launch_mx_settle(h, 0);
    launch_mx_outer(h, 2);
    launch_mx_settle(h, 1);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h.h_ds, h.ds, sizeof(DevState), cudaMemcpyDeviceToHost, h.stream));
  if (e_hist && n > 0) CK(cudaMemcpyAsync(e_hist, h.e_hist, (size_t)n * 8, cudaMemcpyDefault, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  h.last_iters = n;
  h.h_ds->done = 1;
  CK(cudaMemcpyAsync(h.ds, h.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  return OCI_OK;
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy a [J][K] ABI array (host or device) into the device SoA array [K][Jp]
static int put_soa(Handle &h, const double *src, double *dst, int K) {
  const size_t bytes = (size_t)h.J * K * 8;
  const double *s = src;
  if (!is_device_ptr(src)) {
    CK(cudaMemcpyAsync(h.stage, src, bytes, cudaMemcpyHostToDevice, h.stream));
    s = h.stage;
  }
  launch_transpose_in(h, s, dst, K);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h.stream));
  return OCI_OK;
}

static int get_soa(const Handle &hc, const double *src, double *dst, int K) {
  Handle &h = const_cast<Handle &>(hc);
  const size_t bytes = (size_t)h.J * K * 8;
  if (is_device_ptr(dst)) {
    launch_transpose_out(h, src, dst, K);
  } else {
    launch_transpose_out(h, src, h.stage, K);
    CK(cudaMemcpyAsync(dst, h.stage, bytes, cudaMemcpyDeviceToHost, h.stream));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h.stream));
  return OCI_OK;
}

__global__ void k_fp64_peak(double *out, int iters) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  const double m = 0.999999, c = 1.0;
  for (int i = 0; i < iters; i++) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

}  // namespace oci

using namespace oci;

#define GUARD(h)                                                                          \
  do {                                                                                    \
    if (!(h)) return set_error("handle is NULL"), OCI_E_INVAL;                            \
    if ((h)->batch) return set_error("not valid on a batched handle"), OCI_E_STATE;      \
  } while (0)

extern "C" {

int oci_setup(const oci_problem *p, oci_handle **out) {
  if (!out) return set_error("out is NULL"), OCI_E_INVAL;
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  oci_handle *h = new (std::nothrow) oci_handle();
  if (!h) return set_error("host allocation failed"), OCI_E_NOMEM;
  rc = setup_impl(p, h);
  if (rc) {
    free_handle(h);
    return rc;
  }
  *out = h;
  set_error("");
  return OCI_OK;
}

int oci_step(oci_handle *h, oci_stats *st) {
  GUARD(h);
  return run_step(*h, false, st);
}

int oci_solve_transient(oci_handle *h, int32_t n_steps, double *phi_out, oci_stats *st) {
  GUARD(h);
  if (n_steps < 0) return set_error("n_steps must be >= 0"), OCI_E_INVAL;
  const size_t per = (size_t)h->J * h->G * 4;
  for (int k = 0; k < n_steps; k++) {
    int rc = run_step(*h, false, st ? st + k : nullptr);
    if (rc) return rc;
    if (phi_out) {
      rc = get_soa(*h, h->phi, phi_out + per * k, h->G * 4);
      if (rc) return rc;
    }
  }
  return OCI_OK;
}

static int ensure_si(Handle &h) {
  if (h.g_si) return OCI_OK;
  if (h.si_z) return build_graph(h, true, &h.g_si);
  const size_t G = h.G, N = h.N, Jp = h.Jp;
  CK(cudaMalloc(&h.si_z, G * N * 4 * Jp * 8));
  CK(cudaMalloc(&h.si_uin, G * N * 2 * Jp * 8));
  CK(cudaMalloc(&h.phi_si[0], G * 4 * Jp * 8));
  CK(cudaMalloc(&h.phi_si[1], G * 4 * Jp * 8));
  const size_t nm = si_scan_maps(h);
  CK(cudaMalloc(&h.si_maps, nm * 6 * 8));
  CK(cudaMalloc(&h.si_segin, nm * 2 * 8));
  return build_graph(h, true, &h.g_si);
}

int si_sweep(oci_handle *h, oci_stats *st) {
  GUARD(h);
  int rc = ensure_si(*h);
  if (rc) return rc;
  return run_step(*h, true, st);
}

int oci_iterate(oci_handle *h, int32_t n, double *e_hist) {
  GUARD(h);
  return run_fixed(*h, false, n, e_hist);
}

int oci_iterate_part(oci_handle *h, int32_t part, double *e_out) {
  GUARD(h);
  if (part != 0 && part != 1) return set_error("part must be 0 or 1"), OCI_E_INVAL;
  if (h->precision != OCI_FP64 || h->solver != OCI_SOLVER_STRUCTURED || h->ordering != OCI_ORDER_JACOBI ||
      h->accel != 0)
    return set_error("oci_iterate_part: FP64 structured solver, Jacobi ordering, no acceleration"), OCI_E_STATE;
  Handle &H = *h;
  if (part == 0) {
    if (H.part_pending) return set_error("oci_iterate_part: part 0 issued twice"), OCI_E_STATE;
    int rc = begin_iteration(H, 1, H.e_hist_cap);
    if (rc) return rc;
    if (!H.tc_fresh) {  // the step constant depends only on psi_{k-1/2}, Q and dt
      launch_step_const(H);
      H.tc_fresh = 1;
    }
    launch_oci_sweep_part(H, 0);
    CK(cudaGetLastError());
    H.part_pending = 1;
    return OCI_OK;
  }
  if (!H.part_pending) return set_error("oci_iterate_part: part 1 without part 0"), OCI_E_STATE;
  H.part_pending = 0;
  launch_oci_sweep_part(H, 1);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(H.h_ds, H.ds, sizeof(DevState), cudaMemcpyDeviceToHost, H.stream));
  if (e_out) CK(cudaMemcpyAsync(e_out, H.e_hist, 8, cudaMemcpyDefault, H.stream));
  CK(cudaStreamSynchronize(H.stream));
  H.last_iters = 1;
  H.h_ds->done = 1;
  CK(cudaMemcpyAsync(H.ds, H.h_ds, sizeof(DevState), cudaMemcpyHostToDevice, H.stream));
  CK(cudaStreamSynchronize(H.stream));
  return OCI_OK;
}

int si_iterate(oci_handle *h, int32_t n, double *e_hist) {
  GUARD(h);
  int rc = ensure_si(*h);
  if (rc) return rc;
  return run_fixed(*h, true, n, e_hist);
}

int oci_get_psi(const oci_handle *h, double *psi) {
  GUARD(h);
  if (!psi) return set_error("psi is NULL"), OCI_E_INVAL;
  return get_soa(*h, h->Psi[h->h_ds->cur], psi, h->G * h->N * 4);
}

int oci_set_psi(oci_handle *h, const double *psi) {
  GUARD(h);
  if (!psi) return set_error("psi is NULL"), OCI_E_INVAL;
  int rc = put_soa(*h, psi, h->Psi[h->h_ds->cur], h->G * h->N * 4);
  if (rc || h->guess != OCI_GUESS_USER) return rc;
  // GUESS_USER: keep the caller's iterate as the initial iterate of every step
  const size_t nPsi = (size_t)h->G * h->N * 4 * h->Jp;
  CK(cudaMemcpyAsync(h->psi_user, h->Psi[h->h_ds->cur], nPsi * 8, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return OCI_OK;
}

int oci_get_phi(const oci_handle *h, double *phi) {
  GUARD(h);
  if (!phi) return set_error("phi is NULL"), OCI_E_INVAL;
  return get_soa(*h, h->phi, phi, h->G * 4);
}

int oci_get_state(const oci_handle *h, double *psi_prev, double *t) {
  GUARD(h);
  if (t) *t = h->t;
  if (!psi_prev) return OCI_OK;
  return get_soa(*h, h->psi_prev, psi_prev, h->G * h->N * 2);
}

int oci_set_state(oci_handle *h, const double *psi_prev, double t) {
  GUARD(h);
  if (!std::isfinite(t)) return set_error("t must be finite"), OCI_E_INVAL;
  h->tc_fresh = 0;
  if (psi_prev) {
    int rc = put_soa(*h, psi_prev, h->psi_prev, h->G * h->N * 2);
    if (rc) return rc;
  }
  h->t = t;
  return OCI_OK;
}

int oci_get_balance(const oci_handle *h, double *bal) {
  GUARD(h);
  if (!bal) return set_error("bal is NULL"), OCI_E_INVAL;
  CK(cudaMemcpyAsync(bal, h->bal, (size_t)h->G * 10 * 8, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return OCI_OK;
}

int oci_set_boundary(oci_handle *h, const double *inc_left, const double *inc_right) {
  GUARD(h);
  const size_t n = (size_t)h->G * h->N * 2;
  std::vector<double> tmp(2 * n, 0.0);
  if (inc_left) CK(cudaMemcpy(tmp.data(), inc_left, n * 8, cudaMemcpyDefault));
  if (inc_right) CK(cudaMemcpy(tmp.data() + n, inc_right, n * 8, cudaMemcpyDefault));
  if (!all_finite(tmp.data(), 2 * n)) return set_error("incident fluxes must be finite"), OCI_E_INVAL;
  CK(cudaMemcpyAsync(h->inc, tmp.data(), 2 * n * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return OCI_OK;
}

int oci_get_e_hist(const oci_handle *h, double *e_hist, int32_t *n) {
  GUARD(h);
  const int cnt = std::min(h->last_iters, h->e_hist_cap);
  if (n) *n = cnt;
  if (e_hist && cnt > 0) {
    CK(cudaMemcpyAsync(e_hist, h->e_hist, (size_t)cnt * 8, cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return OCI_OK;
}

int oci_set_ordering(oci_handle *h, int32_t ordering) {
  GUARD(h);
  if (ordering != OCI_ORDER_JACOBI && ordering != OCI_ORDER_RED_BLACK)
    return set_error("bad ordering"), OCI_E_INVAL;
  if (ordering == OCI_ORDER_RED_BLACK &&
      !((h->precision == OCI_FP64 && h->solver != OCI_SOLVER_DENSE_LU) || h->precision == OCI_FP32_IR))
    return set_error("red-black ordering needs the FP64 structured solver or the FP32_IR form"), OCI_E_INVAL;
  if (ordering == h->ordering) return OCI_OK;
  if (ordering == OCI_ORDER_RED_BLACK && h->accel != OCI_ACCEL_NONE)
    return set_error("red-black ordering and GMRES acceleration do not combine"), OCI_E_INVAL;
  if (ordering == OCI_ORDER_RED_BLACK && !h->rb_tuned) {  // FP64: time the red-black shapes once
    int rc = tune_rb64(*h);
    if (rc) return rc;
    h->rb_tuned = true;
  }
  const int previous = h->ordering;
  h->ordering = ordering;
  if (h->precision == OCI_FP32_IR) {
    int rc = ordering == OCI_ORDER_RED_BLACK ? tune_rb(*h) : OCI_OK;
    if (rc) {
      h->ordering = previous;
      return rc;
    }
    if (ordering == OCI_ORDER_JACOBI) {  // back to the Jacobi inner sweep tuned at setup
      h->mx_kind = h->mx_jac_kind;
      h->mx_cb = h->mx_jac_cb;
      h->mx_P = h->mx_jac_P;
    }
  }
  if (h->g_oci) {
    cudaGraphExecDestroy(h->g_oci);
    h->g_oci = nullptr;
  }
  return build_graph(*h, false, &h->g_oci);
}

int oci_set_acceleration(oci_handle *h, int32_t accel, int32_t restart, double residual_factor) {
  GUARD(h);
  if (accel != OCI_ACCEL_NONE && accel != OCI_ACCEL_GMRES) return set_error("bad acceleration"), OCI_E_INVAL;
  if (accel == OCI_ACCEL_GMRES) {
    if (h->precision != OCI_FP64 || h->solver == OCI_SOLVER_DENSE_LU || h->ordering != OCI_ORDER_JACOBI)
      return set_error("GMRES acceleration needs the FP64 structured solver in Jacobi order"), OCI_E_INVAL;
    if (restart < 1 || restart > 32) return set_error("restart must be in [1, 32]"), OCI_E_INVAL;
    if (!(residual_factor > 0.0) || residual_factor > 1.0)
      return set_error("residual_factor must be in (0, 1]"), OCI_E_INVAL;
    if (restart != h->gm_restart) gmres_free(*h);  // storage is sized by the restart length
    h->gm_restart = restart;
    h->gm_factor = residual_factor;
  }
  h->accel = accel;
  return OCI_OK;
}

int oci_set_si_mode(oci_handle *h, int32_t mode) {
  GUARD(h);
  if (mode != OCI_SI_SEQUENTIAL && mode != OCI_SI_SCAN) return set_error("bad SI mode"), OCI_E_INVAL;
  if (mode == h->si_mode) return OCI_OK;
  h->si_mode = mode;
  if (h->g_si) {
    cudaGraphExecDestroy(h->g_si);
    h->g_si = nullptr;
    return build_graph(*h, true, &h->g_si);
  }
  return OCI_OK;
}

int oci_get_edges(const oci_handle *hc, double *left, double *right) {
  GUARD(hc);
  Handle &h = const_cast<oci_handle &>(*hc);
  const int K = h.G * h.N;
  const double *P = h.Psi[h.h_ds->cur];
  launch_edges(h, P, h.stage);  // stage[0:2K] = left, stage[2K:4K] = right
  CK(cudaGetLastError());
  if (left) CK(cudaMemcpyAsync(left, h.stage, (size_t)2 * K * 8, cudaMemcpyDefault, h.stream));
  if (right) CK(cudaMemcpyAsync(right, h.stage + 2 * K, (size_t)2 * K * 8, cudaMemcpyDefault, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  return OCI_OK;
}

int oci_commit(oci_handle *h, oci_stats *st) {
  GUARD(h);
  h->tc_fresh = 0;  // the carry writes psi_{k-1/2}
  h->h_ds->status = OCI_OK;
  h->h_ds->done = 1;
  CK(cudaMemcpyAsync(h->ds, h->h_ds, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  launch_carry(*h);
  CK(cudaMemcpyAsync(h->h_bal, h->bal, (size_t)h->G * 10 * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  h->t += h->dt;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->t = h->t;
    for (int g = 0; g < h->G; g++)
      for (int b = 0; b < 2; b++) {
        const double *x = h->h_bal + g * 10 + b * 5;
        const double r = x[0] + x[1] + x[2] - x[3] - x[4];
        const double sc = fabs(x[0]) + fabs(x[1]) + fabs(x[2]) + fabs(x[3]) + fabs(x[4]);
        const double rel = sc > 0 ? fabs(r) / sc : 0.0;
        if (rel > st->balance_rel[b]) st->balance_rel[b] = rel;
      }
  }
  return OCI_OK;
}

int oci_get_info(const oci_handle *h, oci_info *info) {
  GUARD(h);
  if (!info) return set_error("info is NULL"), OCI_E_INVAL;
  info->n_types = h->tt.n_types;
  if (h->precision == OCI_FP64) {
    SweepCfg c = sweep_config(*h);
    info->cells_per_block = c.cells_per_block;
    info->angle_chunks = c.chunks;
    info->inner_kernel = -1;
  } else if (h->precision == OCI_FP32_IR) {
    int cb = 0, P = 0;
    mx_shape(*h, cb, P);
    info->cells_per_block = cb;
    info->angle_chunks = P;
    info->inner_kernel = h->mx_kind;
  } else {
    info->cells_per_block = 128;
    info->angle_chunks = 1;
    info->inner_kernel = 2;
  }
  info->tuned_sweep_us = h->tune_us;
  info->sweep_kernel = h->precision == OCI_FP64 && h->solver != OCI_SOLVER_DENSE_LU ? (h->tune_reg ? 1 : 0) : -1;
  if (info->sweep_kernel >= 0 && h->ordering == OCI_ORDER_RED_BLACK) {
    if (!h->rb_pingpong) {
      info->sweep_kernel = 4;
    } else if (h->rb_cb > 0) {
      info->sweep_kernel = h->rb_reg ? 3 : 2;
      info->cells_per_block = h->rb_cb;
      info->angle_chunks = h->rb_P;
      info->tuned_sweep_us = h->rb_tune_us;
    } else {
      info->sweep_kernel = 2;
    }
  }
  info->multi_sweep = info->sweep_kernel != 1 ? 0 : sweep_cl_grid(*h) > 0 ? 2 : sweep_ms_grid(*h) > 0 ? 1 : 0;
  return OCI_OK;
}

void oci_destroy(oci_handle *h) { free_handle(h); }

const char *oci_last_error(void) { return g_err.c_str(); }

int oci_probe_fp64_peak(double *flops_per_s) {
  if (!flops_per_s) return set_error("NULL argument"), OCI_E_INVAL;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  double *out = nullptr;
  CK(cudaMalloc(&out, (size_t)blocks * threads * 8));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  k_fp64_peak<<<blocks, threads>>>(out, 64);
  float best = 1e30f;
  for (int r = 0; r < 3; r++) {
    cudaEventRecord(a);
    k_fp64_peak<<<blocks, threads>>>(out, iters);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "fp64 peak probe");
  *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3);
  return OCI_OK;
}

}  // extern "C"
