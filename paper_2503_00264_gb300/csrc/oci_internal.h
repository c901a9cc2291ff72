// oci_internal.h -- shared declarations of liboci (not part of the ABI).
//
// Device layout (structure of arrays, cells fastest so that consecutive threads
// touch consecutive addresses):
//   Psi, tc      [G][N][4][Jp]   element (g,m,p,j) at ((g*N+m)*4+p)*Jp + j
//   psi_prev     [G][N][2][Jp]
//   phi, Q       [G][4][Jp]
// Jp = J rounded up to a multiple of 32.  The ABI's [J][G][N][*] order is
// converted by transpose kernels in oci_api.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <string>
#include <vector>

#include "../../include/oci.h"

namespace oci {

constexpr int kMaxN = 128;
constexpr int kMaxG = 16;
constexpr int kMaxUnknowns = 2048;      // 4*N*G per cell
constexpr int kFinalizeThreads = 512;

// Test and profiling overrides.  liboci reads its OCI_* environment variables
// (a pinned kernel or launch shape, no graph, the autotuner off, a short
// device spin limit, ...) only when OCI_TEST_HOOKS=1 is set as well; otherwise
// every override is ignored, so a caller's environment cannot change which
// code runs.  The variables are listed in include/oci.h.
inline const char *hook_env(const char *name) {
  const char *on = getenv("OCI_TEST_HOOKS");
  if (!on || on[0] != '1' || on[1] != 0) return nullptr;
  return getenv(name);
}

// Iterations of the bounded grid-barrier spin of the cooperative multi-sweep
// kernels (each iteration sleeps ~64 ns); OCI_TEST_SPIN_LIMIT lowers it.
constexpr long long kGridSpin = 1 << 21;

// Device-resident iteration state of one handle.
struct DevState {
  int cur;        // index (0/1) of the Psi buffer holding the current iterate
  int l;          // sweeps done in this step
  int status;     // OCI_OK while iterating / converged, OCI_E_NOCONV, OCI_E_NONFINITE
  int done;       // 1 once the stop rule (or a failure) ended the loop
  int max_iter;
  int fixed;      // 1: no stop test (oci_iterate)
  double tol;
  double e, e_prev, rho;
  // mixed-precision form (inner sweeps on an FP32 correction, FP64 refinement)
  int dcur;       // index (0/1) of the delta buffer holding the current correction
  int blk_i;      // inner sweeps since the last refinement (0: correction is zero)
  int refine;     // 1: the next outer kernel applies delta and refreshes the residual
  int applied;    // 1: the correction has been folded into Psi after convergence
  int k_max;      // inner sweeps per refinement at most
  int n_refine;   // refinements in this step
  double theta;   // refine once e < theta * (first e of the block)
  double e_blk0;
  int inplace;    // 1: the sweep updates Psi[cur] in place (red-black ordering)
  unsigned long long cond_ref;  // mixed forms in a graph: handle of the IF node of the refinement
  long long spin;               // grid-barrier spin limit of the cooperative kernels (kGridSpin)
};

// Per-cell-type tables of the structured solve (all FP64, device).
struct TypeTables {
  int n_types = 0;
  double *Linv = nullptr;   // [T][G][N][16]  inverse of the 4x4 L_{c,g,m} (Eq. Aj), row-major
  double *Cin = nullptr;    // [T][G][N][8]   |mu| * the two columns of Linv that the inflow feeds
  double *Win = nullptr;    // [T][G][N][8]   w_m * Cin (the inflow's part of y)
  double *Mp = nullptr;     // [T][4G][4G]    s = Mp y: within-cell scattering source from y
  double *Kap = nullptr;    // [T][G][G]      dx/4 * Sigma_s,gp->g  (index [gp][g])
  double *dx = nullptr;     // [T]
  double *sig = nullptr;    // [T][G]         Sigma_t,g
  double *Lco = nullptr;    // [T][G][N][5]   {a, mu/2, alpha/2, alpha, alpha+a} of L_{c,g,m} (Eq. Aj)
  float *Linv32 = nullptr;  // FP32 copies for the low-precision inner solve
  float *Cin32 = nullptr;
  float *Mp32 = nullptr;
};

struct Batch;

struct Handle {
  Batch *batch = nullptr;          // set on handles made by oci_batch_setup
  int J = 0, N = 0, G = 0, n_mat = 0, Jp = 0;
  double dt = 0, tol = 0, t = 0;
  int max_iter = 0, precision = 0, guess = 0, solver = 0;
  int ordering = OCI_ORDER_JACOBI;  // cell ordering of the FP64 structured sweep
  cudaStream_t stream = nullptr;
  int device = 0;

  // host copies of the problem (for re-setup and validation)
  std::vector<double> h_dx, h_sigma_t, h_sigma_s, h_v;
  std::vector<int32_t> h_mat;
  std::vector<double> h_mu, h_w;
  std::vector<int32_t> h_type;   // cell -> type

  // device state
  double *Psi[2] = {nullptr, nullptr};
  double *tc = nullptr;          // per-step constant Linv * c (structured) or c (dense)
  double *yc = nullptr;  // [G][4][Jp] yc = sum_m w_m tc (per step; register sweep)
  double *psi_prev = nullptr;
  double *phi = nullptr;
  double *phi_si[2] = {nullptr, nullptr};
  double *Q = nullptr;
  double *inc = nullptr;         // [2][G][N][2] left, right
  int32_t *type = nullptr;       // [Jp]
  double *mu = nullptr, *w = nullptr, *v = nullptr;
  TypeTables tt;
  // mixed-precision form
  float *delta[2] = {nullptr, nullptr};  // [G][N][4][Jp] correction ping-pong
  float *z32 = nullptr;                  // [G][N][4][Jp] L~^{-1} r of the last refinement
  float *w32 = nullptr;
  float *mu32 = nullptr;           // mixed forms: FP32 copy of the ordinates
  int mx_kmax = 128;
  double mx_theta = 1e-4;
  CUtensorMap tm_z, tm_d[2];          // TMA descriptors of z32 and delta[0/1] ([R][Jp] FP32)
  bool tma_ok = false;                 // tensor maps encoded (4NG <= 256)
  CUtensorMap tm_bg_r, tm_bg_d[2];     // tensor-core form, 4NG > 128: r and correction boxes of 32 rows
  unsigned long long mx_cond_ref = 0;  // IF-node handle of the refinement in the mixed-form graph
  int mx_jac_kind = 0, mx_jac_cb = 0, mx_jac_P = 0;  // the Jacobi FP32 inner sweep (kept while red-black)
  int mx_tune_sweeps = 0;              // > 0 while the autotuner times a multi-sweep launch of that many sweeps
  bool mx_multi = true;                // graph runs the persistent tiled FP32 sweep several sweeps per launch
  bool rb_pingpong = true;             // FP64 red-black: ping-pong buffers (false: in place)
  int rb_cb = 0, rb_P = 0;             // FP64 red-black shape timed at setup (0: the Jacobi staged shape)
  bool rb_reg = false;                 // that shape is the register form
  double rb_tune_us = 0.0;             // its timed sweep (both colours), microseconds
  bool rb_tuned = false;               // red-black shapes timed (on the first switch to red-black)
  int mx_hwcvt = 0;                    // 1: FP64 refinement converts with the compiler's F2F (same bits, slower)
  unsigned *gbar = nullptr;            // two words: the 64-bit arrival count of the cooperative kernels' grid barrier
  int mx_kind = 0;                     // FP32 inner sweep picked by the autotuner: kMxPlain, kMxTma, kMxReg, kMxTiled
  unsigned char *tc_img = nullptr;     // [T] x (A^{-1} image(s) in the tcgen05 K-major layout)
  size_t tc_img_bytes = 0;             // bytes per type
  unsigned char *tc_img_h = nullptr;   // [T] x image of A~^{-1} B: the inflow columns, |mu| folded in (k_tc_big)
  float *tc_z = nullptr;               // [R][Jp] z = A~^{-1} r of the current refinement block (k_tc_big)
  int2 *tc_items = nullptr;            // streamed tcgen05 apply: (tile, cell type) work items
  int tc_n_items = 0;
  bool tc_mixed = false;               // some 128-cell tile holds more than one cell type
  // SI scratch
  double *si_z = nullptr;        // [G][N][4][Jp]   Linv * d0
  double *si_uin = nullptr;      // [G][N][2][Jp]   incoming edge of every cell
  double *si_maps = nullptr;     // [G*N][K][6]     scan form: segment affine maps
  double *si_segin = nullptr;    // [G*N][K][2]     scan form: incoming edge of each segment
  int si_mode = 0;               // 0 sequential chain (the paper's SI), 1 scan form
  // dense path
  double *LU = nullptr;          // [J][n][n] column-major per cell: A_j^{-1} (dense_inv) or its LU factors
  int32_t *piv = nullptr;        // [J][n] (LU factors only)
  int dense_inv = 1;             // 1: apply the explicit inverse; 0: triangular solves with the LU factors
  // reductions
  double *partials = nullptr;    // [max blocks]
  unsigned *counter = nullptr;   // blocks finished in the current sweep launch (last block resets it)
  int n_partials = 0;
  double *bal_partials = nullptr;  // [max blocks][G][8]
  double *bal = nullptr;           // [G][2][5]
  double *e_hist = nullptr;        // [e_hist_cap]
  int e_hist_cap = 0;
  double *stage = nullptr;         // device staging buffer, size of one Psi
  double *psi_user = nullptr;      // GUESS_USER: the caller's initial iterate (device SoA)
  DevState *ds = nullptr;
  // pinned host mirrors
  DevState *h_ds = nullptr;
  double *h_bal = nullptr;
  // graphs
  cudaGraphExec_t g_oci = nullptr, g_si = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int last_iters = 0;
  int part_pending = 0;  // oci_iterate_part: part 0 issued, part 1 not yet
  int tc_fresh = 0;      // oci_iterate_part: tc holds this step's constant (cleared by any other
                         // path that runs sweeps, commits or sets the state)
  bool no_graph = false;           // OCI_NO_GRAPH=1: host-driven loop instead of the WHILE graph
  int tune_cb = 0, tune_P = 0;     // sweep launch shape picked by the autotuner (0: default)
  bool tune_reg = false;           // FP64 Jacobi sweep in the register form (k_oci_sweep_reg)
  // Krylov acceleration of the FP64 step (OCI_ACCEL_GMRES): restart length, residual
  // factor (stop when ||F(x) - x|| < tol * factor) and device storage
  int accel = 0, gm_restart = 20;
  double gm_factor = 0.05;
  double *gm_V = nullptr, *gm_w = nullptr, *gm_zero = nullptr, *gm_part = nullptr, *gm_h = nullptr;
  DevState *gm_ds = nullptr;
  int mx_cb = 0, mx_P = 0;         // same for the FP32 inner sweep of the mixed form
  double tune_us = 0.0;            // measured sweep time of the chosen shape
};

// ---------------------------------------------------------------- launches
struct SweepCfg {
  int cells_per_block;
  int chunks;  // angle chunks per (cell, group): threads per cell and group
  int grid;
  size_t smem;
};
SweepCfg sweep_config(const Handle &h);
size_t sweep_smem(int N, int G, int cb, int P, size_t es);

void launch_step_const(Handle &h);
void launch_oci_apply(Handle &h, const double *in, double *out, const double *tc, const double *inc,
                      DevState *ds_apply);
int gmres_solve(Handle &h, double tol_g, int max_sweeps, int &sweeps, double &e_last, int &status);
void gmres_free(Handle &h);
void launch_oci_sweep(Handle &h, cudaGraphConditionalHandle cond, int use_cond);
int sweep_ms_grid(const Handle &h);
int sweep_cl_grid(const Handle &h);
void launch_oci_sweep_cl(Handle &h, int grid, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps);
void launch_oci_sweep_ms(Handle &h, int grid, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps);
void launch_oci_sweep_part(Handle &h, int part);  // FP64 Jacobi sweep as interior (0) and end blocks (1)
const void *k_oci_sweep_ptr();
const void *k_oci_sweep_rb_ptr();
const void *k_oci_sweep_rbpp_ptr();
int sweep_partials(const Handle &h);
void launch_finalize(Handle &h, const double *partials, int n, cudaGraphConditionalHandle cond,
                     int use_cond);
void launch_carry(Handle &h);
void launch_transpose_in(Handle &h, const double *src_abi, double *dst_soa, int P);
void launch_transpose_out(Handle &h, const double *src_soa, double *dst_abi, int P);
void launch_phi_out(Handle &h, double *dst_abi);
void launch_edges(Handle &h, const double *Psi, double *out);
// SI
void launch_si_sweep(Handle &h);
void launch_si_phi_from_psi(Handle &h, double *phi_dst);
size_t si_scan_maps(const Handle &h);
// mixed-precision form
void launch_mx_inner(Handle &h, cudaGraphConditionalHandle cond, int use_cond);
void launch_mx_outer(Handle &h, int mode);
void launch_mx_finalize(Handle &h, cudaGraphConditionalHandle cond, int use_cond);
int mx_partials(const Handle &h);
int mx_tma_setup(Handle &h);
// FP32 inner sweeps of the mixed form (values of Handle::mx_kind and oci_info.inner_kernel);
// kMxTiled, kMxTiledP (persistent), kMxTiledB (persistent, tiles moved by
// 1D bulk copies) and kMxRB (red-black ordering, columns of a tile ordered by
// colour) keep the FP32 correction arrays tile-major
// ([J/T][4NG][T], T = mx_cb)
constexpr int kMxPlain = 0, kMxTma = 1, kMxReg = 3, kMxTiled = 4, kMxTiledP = 5, kMxTiledB = 6, kMxRB = 7;
constexpr int kSweepReg64 = 8;  // autotuner candidate kind of the FP64 register sweep
constexpr int kMxTiled2 = 9;    // tile-major, two inner sweeps per pass (temporal blocking)
constexpr int kMxTiled2Occ = 10;  // the same built for more resident blocks per SM (S16, one group)
constexpr int kMxRB2 = 11;        // red-black ordering, two sweeps per pass (colour-ordered tiles)
constexpr int kMxWarp2 = 12;      // tile-major, two sweeps per pass, one run of cells per warp (one group)
size_t mx_rb2_smem(const Handle &h, int T, int P, bool stage);
// two-sweep-per-pass inner kernels (oci_mixed_two.cu, oci_mixed_rb2.cu)
void launch_ms2_any(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps);
void launch_rb2_any(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps);
int mx_two_set_attributes();
int mx_rb2_set_attributes();
// warp-run two-sweep inner kernel (oci_mixed_warp.cu): one group, N = 8, 16, 32
bool mx_w2_supported(const Handle &h);
void launch_w2_any(Handle &h, cudaGraphConditionalHandle cond, int use_cond, int max_sweeps);
int mx_w2_set_attributes();
size_t mx_ms2_smem(const Handle &h, int T, int P, bool stage);
size_t mx_tb_smem(const Handle &h, int T, int P, bool stage);
size_t mx_tables_floats(const Handle &h);
int mx_tile_shift(const Handle &h);
int mx_set_attributes();
size_t sweep_reg_smem(int G, int cb, int P);
const void *k_oci_sweep_reg_ptr(int np);
void mx_shape(const Handle &h, int &cb, int &P);
size_t mx_tma_smem(const Handle &h, int P);
// tensor-core block apply (TF32 / BF16x3 forms)
int tc_prepare(Handle &h);
bool tc_pipe_ok(const Handle &h);
void launch_tc_pipe(Handle &h, cudaGraphConditionalHandle cond, int use_cond);
int tc_partials(const Handle &h);
void launch_tc_inner(Handle &h);
int tc_build_images(Handle &h, const std::vector<double> &Ainv);
// tensor-core form for 128 < 4NG <= 512 (oci_tc_big.cu)
bool tc_big_used(const Handle &h);
int tc_big_prepare(Handle &h);
void launch_tc_big(Handle &h, cudaGraphConditionalHandle cond, int use_cond);
int tc_big_build_images(Handle &h, const std::vector<double> &Ainv, float (*round_tf32)(float),
                        uint16_t (*bf16_bits)(float), float (*bf16_value)(uint16_t));
// dense path
int dense_setup(Handle &h);
void launch_dense_step_const(Handle &h);
void launch_dense_sweep(Handle &h);

// errors
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// setup helpers shared with the batched form
int validate(const oci_problem *p);
void gauss_legendre(int N, std::vector<double> &x, std::vector<double> &wt);
int build_tables(Handle &h, std::vector<double> &Linv, std::vector<double> &Cin, std::vector<double> &Mp,
                 std::vector<double> &Kap, std::vector<double> &tdx, std::vector<double> &tsig,
                 std::vector<double> &Lco);

}  // namespace oci

struct oci_handle : public oci::Handle {};
