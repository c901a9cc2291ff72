/*
 * oci.h -- C ABI of liboci: one-cell inversion (OCI) and source iteration (SI)
 * for the simple-corner-balance (SCB) x multiple-balance (MB) discretisation of
 * time-dependent multigroup slab S_N transport, on NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2503.00264 (Morgan, Variansyah, Palmer, Niemeyer).
 *   problem statement ............. Sec. 2.1, Eq. sn_nte
 *   space-time discretisation ..... Eqs. scb-mb-a..d and the two closures
 *   per-cell OCI system ........... Eqs. oci, Aja, Aj, rhs_sg, scatter, x_vec
 *   multigroup system ............. Sec. 2.4, Eqs. scatter_mg, fullOCIlhs/rhs
 *   stop rule ..................... Sec. 2.1 (||Psi^{l+1}-Psi^l||_2 < eps(1-rho_e))
 *   OCI loop ...................... Algorithm 2
 *   SI loop ....................... Algorithm 1, App. A
 *
 * Conventions shared by every entry point
 *   - Every function returns int status: OCI_OK (0) or a negative OCI_E_* code;
 *     oci_last_error() then gives a message (thread-local).  No C++ exception
 *     crosses the ABI.
 *   - Arrays are dense, row-major (C order), FP64 unless stated otherwise.
 *   - Array arguments marked "host or device" may be host memory (pageable or
 *     pinned) or CUDA device memory of the handle's device; the library copies
 *     with cudaMemcpyAsync(..., cudaMemcpyDefault) on the handle's stream and
 *     synchronises that stream before returning.
 *   - Ownership: the caller owns every array it passes; oci_setup copies what it
 *     needs, so inputs may be freed once it returns.  The library owns the
 *     handle and all device memory behind it; oci_destroy releases them.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Invalid arguments return OCI_E_INVAL before any device work.
 *   - Angles are Gauss-Legendre ordinates in ascending mu (the first N/2 are
 *     negative), with weights summing to 2.
 *   - Unknowns of one cell are ordered idx(g,m,p) = (g*N + m)*4 + p with
 *     p = 0 kL, 1 kR, 2 hL, 3 hR (k: time average over the step, h: time edge
 *     t_{k+1/2}; L/R: left/right corner) -- Eq. x_vec extended to groups.
 *   - The environment does not change what runs.  For tests and profiling the
 *     library honours these variables, read at setup (the spin limit at every
 *     step), only when OCI_TEST_HOOKS=1 is also set:
 *       OCI_AUTOTUNE=0            keep the default launch shapes (no timing)
 *       OCI_SWEEP_SHAPE=cb,P      pin the sweep shape (cells per block, angle chunks)
 *       OCI_SWEEP_REG=0|1         FP64 sweep: staged or register form only
 *       OCI_SWEEP_MS=0|grid       FP64 register form in the graph: one launch per sweep, or
 *                                 the cooperative all-sweeps launch but not the cluster one
 *       OCI_MX_INNER=plain|tma|reg|tiled|tiledp|tiledb|two|twoocc|warp (or a comma list)
 *                                 FP32 inner sweep kernel of the mixed form
 *       OCI_MX_RB=1|2             red-black FP32 inner sweep, one or two sweeps per pass
 *       OCI_MX_MULTI=0            one inner sweep per launch in the graph
 *       OCI_MX_KMAX, OCI_MX_THETA refinement schedule of the mixed forms
 *       OCI_MX_OUTER_CVT=hw       compiler conversions in the FP64 refinement
 *       OCI_RB_FP64=inplace       FP64 red-black half sweeps in place
 *       OCI_RB_SHAPE=s|r,cb,P     pin the FP64 red-black shape
 *       OCI_TC_BIG=0              tensor-core forms at 4NG <= 128: the persistent kernel with
 *                                 the inverse resident in shared memory (not the streamed one)
 *       OCI_TC_PIPE=0             with OCI_TC_BIG=0: the one-tile-per-CTA tensor-core kernel
 *       OCI_TC_HALF=0             streamed tensor-core kernel: the full form r + B delta for
 *                                 every inner sweep (not z + (A~^{-1} B) u after the first)
 *       OCI_DENSE_APPLY=lu        dense per-cell path: triangular solves with the LU
 *                                 factors instead of the explicit inverse
 *       OCI_BATCH_SWEEP           pin the batched sweep form
 *       OCI_NO_GRAPH=1            host-driven loop instead of the CUDA graph
 *       OCI_TEST_SPIN_LIMIT=k     grid-barrier spin limit of the cooperative
 *                                 kernels (0: the step ends with OCI_E_TIMEOUT)
 */
#ifndef OCI_H
#define OCI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
  OCI_OK = 0,
  OCI_E_INVAL = -1,     /* bad argument (detected before any device work)      */
  OCI_E_NOMEM = -2,     /* device or host allocation failed                     */
  OCI_E_CUDA = -3,      /* a CUDA call failed; see oci_last_error()             */
  OCI_E_NOCONV = -4,    /* max_iter sweeps without meeting the stop rule; the
                           step is NOT committed (t and psi_{k-1/2} unchanged,
                           the last iterate stays readable)                     */
  OCI_E_SINGULAR = -5,  /* a local block could not be factored                  */
  OCI_E_NONFINITE = -6, /* the convergence norm became NaN or Inf               */
  OCI_E_TIMEOUT = -7,   /* a bounded device-side wait gave up                   */
  OCI_E_STATE = -8      /* call not valid in the handle's current state         */
};

/* arithmetic of the OCI cell solve (oci_problem.precision) */
enum {
  OCI_FP64 = 0,       /* everything in IEEE FP64                                   */
  OCI_TF32_IR = 1,    /* block apply on tensor cores in TF32 (FP32 accumulation),
                         FP64 residual, norm, balance and carry (defect correction) */
  OCI_BF16X3_IR = 2,  /* block apply as three BF16 products (hi*hi + hi*lo + lo*hi),
                         FP32 accumulation, FP64 residual/norm/balance/carry        */
  OCI_FP32_IR = 3     /* structured block apply in FP32 on the CUDA cores, FP64
                         residual/norm/balance/carry                               */
};
/* The three *_IR forms run the OCI sweeps on an FP32 correction delta of an FP64
 * iterate Psi (delta^{i+1} = A~^{-1}(r + B delta^i), r = c + B Psi - A Psi in
 * FP64) and fold delta into Psi with a fresh FP64 residual every few sweeps
 * (defect correction).  In exact arithmetic the iterates, and so the norm and
 * the stop rule, are those of the FP64 form; the fixed point is the FP64 one.
 * The tensor-core forms (TF32_IR, BF16X3_IR) keep one dense inverse per cell
 * type (4NG <= 512) and apply it to tiles of 128 consecutive cells; a tile with
 * several cell types is taken once per type.  oci_setup returns OCI_E_INVAL
 * when that would more than double the tiles' work or the inverses would
 * exceed 2^28 entries (cell types that change from cell to cell). */

/* initial iterate of every time step (oci_problem.guess) */
enum {
  OCI_GUESS_PREV = 0, /* the handle's current Psi: the previous step's converged
                         Psi, zero before the first step, or what oci_set_psi set */
  OCI_GUESS_ZERO = 1, /* zero                                                      */
  OCI_GUESS_USER = 2  /* the iterate the caller last passed to oci_set_psi (zero
                         before the first call), restored at the start of every
                         step; the handle keeps a device copy of it              */
};

/* local solver of the FP64 form (oci_problem.solver) */
enum {
  OCI_SOLVER_AUTO = 0,       /* structured solve                                  */
  OCI_SOLVER_STRUCTURED = 1, /* exact solve of A_j through its angle blocks and a
                                4G x 4G scalar-flux system per cell type; cells
                                that share (material, dx) share the tables        */
  OCI_SOLVER_DENSE_LU = 2    /* (4NG <= 1024) dense A_j of every cell factored once on the GPU
                                (warp-cooperative LU, partial pivoting), then one
                                forward/back substitution per cell per sweep:
                                the paper's gesv/getrs scheme (Algorithm 2)       */
};

/* cell ordering of the sweeps (oci_set_ordering) */
enum {
  OCI_ORDER_JACOBI = 0,    /* block Jacobi: every cell from the previous iterate (Eq. oci)  */
  OCI_ORDER_RED_BLACK = 1  /* cell-wise block Gauss-Seidel in red-black order (the other
                              OCI ordering the paper names, Sec. 1): even cells from the
                              previous iterate, then odd cells from the new even cells;
                              one sweep = both halves                                      */
};

/* how si_sweep / si_iterate march through the cells (oci_set_si_mode) */
enum {
  OCI_SI_SEQUENTIAL = 0,  /* the paper's SI: each (g,m) sweeps the cells one after another
                             (Algorithm 1), here one GPU thread per (g,m) fed from shared memory */
  OCI_SI_SCAN = 1         /* the same sweep as a parallel scan: the outgoing edge of a cell is
                             an affine function of its incoming edge, affine maps compose
                             associatively, so segments of cells are composed in parallel, the
                             segment maps are scanned, and every segment is walked again from
                             its incoming edge (identical result up to rounding)              */
};

/* Problem description -- the arguments of Eq. sn_nte plus the iteration
 * controls of Sec. 2.1.  Sizes: J cells, N ordinates, G groups. */
typedef struct {
  int32_t J, N, G, n_mat;   /* J >= 1; N even, 2 <= N <= 128; 1 <= G <= 16;
                               4*N*G <= 2048; n_mat >= 1                              */
  const double *dx;         /* [J] cell widths, finite and > 0                        */
  const int32_t *mat;       /* [J] material of each cell, in [0, n_mat)               */
  const double *sigma_t;    /* [n_mat][G] total cross section, >= 0                   */
  const double *sigma_s;    /* [n_mat][G][G]; sigma_s[m][gp][g] = Sigma_s,gp->g >= 0  */
  const double *v;          /* [G] speeds, > 0                                        */
  const double *Q;          /* [J][G][4] isotropic total emission per corner and time
                               level (kL,kR,hL,hR); the angular source is Q/2.
                               NULL = no source                                       */
  double dt;                /* time step, finite and > 0                              */
  const double *psi_init;   /* [J][G][N][2] psi at t = 0 at corners (L,R); NULL = 0   */
  const double *inc_left;   /* [G][N][2] incident flux at x = 0 for mu > 0: index 0 the
                               time average over the step, 1 the value at t_{k+1/2};
                               entries of mu < 0 are ignored.  NULL = vacuum          */
  const double *inc_right;  /* [G][N][2] same at x = X for mu < 0.  NULL = vacuum     */
  double tol;               /* eps of the stop rule, >= 0 (absolute 2-norm)           */
  int32_t max_iter;         /* >= 1 sweeps per step                                   */
  int32_t precision;        /* OCI_FP64 | OCI_TF32_IR | OCI_BF16X3_IR | OCI_FP32_IR   */
  int32_t guess;            /* OCI_GUESS_PREV | OCI_GUESS_ZERO | OCI_GUESS_USER       */
  int32_t solver;           /* OCI_SOLVER_*                                           */
  void *stream;             /* cudaStream_t for all work of the handle; NULL = the
                               legacy default stream                                 */
} oci_problem;

/* Per-step statistics. */
typedef struct {
  int32_t iters;            /* sweeps taken in this step                              */
  int32_t status;           /* OCI_OK or OCI_E_NOCONV / OCI_E_NONFINITE               */
  double e_last;            /* ||Psi^{l+1} - Psi^l||_2 of the last sweep (FP64)       */
  double rho_e_last;        /* e_l / e_{l-1} of the last sweep (0 if l = 0)           */
  double balance_rel[2];    /* max over groups of |balance residual| / sum of |terms|:
                               [0] time-average balance (Eqs. scb-mb-a + b summed),
                               [1] time-edge balance (Eqs. scb-mb-c + d summed)       */
  double t;                 /* simulated time after the step                          */
  double seconds;           /* wall time of the convergence loop (CUDA events)        */
  int32_t refinements;      /* mixed forms: passes of the FP64 refinement that fold the
                               correction into Psi (the last one at convergence; the
                               initial residual not counted); 0 for FP64 and SI      */
  int32_t reserved;
} oci_stats;

/* Setup facts of a handle (oci_get_info). */
typedef struct {
  int32_t n_types;           /* distinct cell types (material, dx) sharing their tables          */
  int32_t cells_per_block;   /* launch shape of the sweep kernel picked by the autotuner         */
  int32_t angle_chunks;      /* threads per (cell, group): angles split into this many chunks    */
  int32_t inner_kernel;      /* mixed forms: 0 plain FP32 sweep, 1 TMA-staged FP32 sweep,
                                2 tcgen05 tensor-core block apply, 3 register FP32 sweep (angles
                                split over threads), 4 the register sweep on tile-major FP32
                                correction arrays, 5 the same as a persistent kernel, 6 that with
                                the tiles moved by 1D bulk copies (TMA), 7 red-black ordering,
                                9 two inner sweeps per pass over the correction (temporal
                                blocking), 10 the same built for more resident blocks per SM,
                                11 red-black ordering with two sweeps per pass, 12 two sweeps per
                                pass with one run of cells per warp (one group); -1 for the FP64
                                form                                                              */
  double tuned_sweep_us;     /* measured time of one sweep with the chosen shape (0 if not tuned) */
  int32_t sweep_kernel;      /* FP64 form: 0 angles staged in shared memory (k_oci_sweep_t),
                                1 angles in registers (k_oci_sweep_reg); red-black order: 2 staged
                                and 3 register form on ping-pong buffers, 4 staged in place;
                                -1 for the other forms                                            */
  int32_t multi_sweep;       /* FP64 Jacobi register form: how the convergence loop runs the
                                sweeps of a step -- 0 one launch per sweep; 1 all in one
                                cooperative launch (every cell block resident at once, a grid
                                barrier between sweeps); 2 all in one thread-block cluster (at
                                most 16 cell blocks, the iterate kept on chip).  Same iterates,
                                norms and sweep counts in all three                              */
} oci_info;

typedef struct oci_handle oci_handle;

/* Validate and copy the problem, build the quadrature and the per-cell-type
 * tables (or the per-cell dense LU factors), move everything to the device.
 * Setup is excluded from the convergence-loop timing, as in the paper
 * (Sec. 3.2).  *out receives a new handle on success. */
int oci_setup(const oci_problem *p, oci_handle **out);

/* One time step (Algorithm 2 and the carry of Sec. 2.1): set the initial
 * iterate per p->guess, sweep until the stop rule holds, then commit: scalar
 * flux, balance tallies, psi_{k+1/2} -> psi_{k-1/2}, t += dt.  The whole
 * convergence loop runs on the device (CUDA graph with a conditional WHILE
 * node; where every cell block of the FP64 register sweep fits on the GPU at
 * once, one launch runs all sweeps: a thread-block cluster with the iterate on
 * chip for up to 16 blocks, else a cooperative grid with a bounded barrier
 * between sweeps); the host reads a small stats record once per step.  st may
 * be NULL.  Returns OCI_E_NOCONV without committing when max_iter is reached,
 * OCI_E_TIMEOUT without committing when a bounded device-side wait gave up. */
int oci_step(oci_handle *h, oci_stats *st);

/* n_steps calls of oci_step.  phi_out: [n_steps][J][G][4] (host or device) or
 * NULL; st: [n_steps] or NULL.  Stops at the first failing step and returns its
 * status. */
int oci_solve_transient(oci_handle *h, int32_t n_steps, double *phi_out, oci_stats *st);

/* The same time step by source iteration (Algorithm 1, App. A): per (g,m)
 * sweep the cells in the direction of flight with the 4x4 L_{c,j,g,m}, the
 * current sweep's upstream edge and the scattering source of all groups lagged
 * from phi^(l) (Jacobi over groups); stop rule on ||phi^{l+1} - phi^l||_2.
 * Commits like oci_step.  Comparison path; FP64 only. */
int si_sweep(oci_handle *h, oci_stats *st);

/* Exactly n OCI (or SI) sweeps from the current iterate, no stop test, no
 * commit; e_hist: [n] (host or device) receives e of each sweep, or NULL.
 * For timing and for parity at a fixed sweep count. */
int oci_iterate(oci_handle *h, int32_t n, double *e_hist);

/* One OCI sweep (Eq. oci, Algorithm 2) in two calls, so that a subdomain can
 * sweep its interior while the lagged edge values of its neighbours are in
 * flight (a spatial decomposition exchanges them before every sweep, Sec. 4):
 * part 0 sweeps the cells of every block but the first and the last -- cells
 * that read no incident flux -- and returns without waiting for the GPU;
 * the caller may then change the incident fluxes (oci_set_boundary); part 1
 * sweeps the first and the last block, forms e = ||Psi^{l+1} - Psi^l||_2 of
 * the whole sweep in the same fixed order as oci_iterate, writes it to e_out
 * (one double, host or device, or NULL) and waits for the GPU.  Together the
 * two parts are oci_iterate(h, 1, e_out) bit for bit.  FP64, structured
 * solver, Jacobi ordering, no acceleration; otherwise OCI_E_STATE, as is part 1
 * without a preceding part 0 and part 0 twice.  e_out is ignored in part 0. */
int oci_iterate_part(oci_handle *h, int32_t part, double *e_out);
int si_iterate(oci_handle *h, int32_t n, double *e_hist);

/* State access.  psi: [J][G][N][4]; phi: [J][G][4]; psi_prev: [J][G][N][2];
 * bal: [G][2][5] = per group, per balance (0 time average, 1 time edge), the
 * tallies {time, leak, collision, scatter_in, source} of the last committed
 * step (residual = time + leak + collision - scatter_in - source).
 * All buffers host or device. */
int oci_get_psi(const oci_handle *h, double *psi);
int oci_set_psi(oci_handle *h, const double *psi); /* with OCI_GUESS_USER also the
                                                      initial iterate of every later step */
int oci_get_phi(const oci_handle *h, double *phi);
int oci_get_state(const oci_handle *h, double *psi_prev, double *t);
int oci_set_state(oci_handle *h, const double *psi_prev, double t);
int oci_get_balance(const oci_handle *h, double *bal);

/* Replace the incident fluxes ([G][N][2] each, host or device, NULL = vacuum)
 * for the following steps. */
int oci_set_boundary(oci_handle *h, const double *inc_left, const double *inc_right);

/* e of every sweep of the last oci_step / si_sweep: e_hist [max_iter] (host or
 * device); *n receives the number of valid entries. */
int oci_get_e_hist(const oci_handle *h, double *e_hist, int32_t *n);

/* Cell ordering of the following OCI sweeps (OCI_ORDER_*; default Jacobi).
 * Red-black needs the FP64 structured solver or the OCI_FP32_IR form and no
 * GMRES acceleration (else OCI_E_INVAL).  The norm and the stop rule are those
 * of Sec. 2.1 over one full (red + black) sweep.  The first switch to red-black
 * times the red-black launch shapes on the handle's stream (the state -- last
 * iterate, psi_{k-1/2}, t -- is left as it was); the switch rebuilds the step's
 * CUDA graph.  Errors leave the ordering unchanged. */
int oci_set_ordering(oci_handle *h, int32_t ordering);

/* March of the following SI sweeps (OCI_SI_*; default sequential). */
int oci_set_si_mode(oci_handle *h, int32_t mode);

/* Edge values for a domain-decomposed driver (Sec. 4 of the paper proposes
 * exchanging them between subdomains every iteration): left [G][N][2] receives
 * (Psi_kL, Psi_hL) of cell 0 -- the inflow a left neighbour needs for mu < 0 --
 * and right [G][N][2] receives (Psi_kR, Psi_hR) of cell J-1 -- the inflow a right
 * neighbour needs for mu > 0.  Either may be NULL; host or device memory. */
int oci_get_edges(const oci_handle *h, double *left, double *right);

/* Commit the current iterate as the converged solution of the step (scalar
 * flux, balance tallies, psi_{k+1/2} -> psi_{k-1/2}, t += dt), for drivers that
 * run the convergence loop themselves through oci_iterate (e.g. across ranks).
 * st may be NULL; st->iters and st->e_last are left 0. */
int oci_commit(oci_handle *h, oci_stats *st);

/* Batched form: n independent slabs (each its own oci_problem: sizes, angle
 * order, groups, materials, dt, tolerances) advanced together.  Slabs that
 * share (N, G) are packed into one cell range; every time step is one CUDA
 * graph launch whose persistent sweep kernels skip slabs that have converged,
 * each slab with its own stop rule (Sec. 2.1).  Precision OCI_FP64, or
 * OCI_FP32_IR (FP32 inner sweeps with per-slab FP64 refinement), one precision
 * for the whole batch; structured solver and OCI_GUESS_PREV only; all problems
 * must name the same stream.  The returned
 * handle accepts only the oci_batch_* calls and oci_destroy (others return
 * OCI_E_STATE). */
int oci_batch_setup(const oci_problem *probs, int32_t n, oci_handle **out);

/* One time step of every slab; st: [n] (or NULL) per-slab statistics.
 * Returns OCI_OK, or the status of a slab that did not converge (that slab is
 * not committed; the others are). */
int oci_batch_step(oci_handle *h, oci_stats *st);

/* Number of slabs of a batched handle. */
int oci_batch_size(const oci_handle *h, int32_t *n);

/* Per-slab state of a batched handle, slab index s in [0, n): psi
 * [J_s][G_s][N_s][4], phi [J_s][G_s][4], bal [G_s][2][5] (as oci_get_balance);
 * host or device memory. */
int oci_batch_get_psi(const oci_handle *h, int32_t s, double *psi);
int oci_batch_get_phi(const oci_handle *h, int32_t s, double *phi);
int oci_batch_get_balance(const oci_handle *h, int32_t s, double *bal);

/* Convergence norm e = ||a - b||_2 over n FP64 values, for callers that cannot
 * allocate device memory when they need it (allocator callbacks, loops whose
 * memory is budgeted once at start-up, applications whose device memory is
 * owned by another framework).  The paper has no counterpart: it is an extra
 * entry point of this library (oci_step computes the same norm internally).
 *   a, b   device pointers to n values each (any layout, same for both)
 *   n      0 <= n <= 33,554,432 (the fixed scratch holds 16,384 partial sums of
 *          2,048 values each); larger n returns OCI_E_INVAL
 *   e_out  device pointer; receives e when the stream reaches it
 *   stream cudaStream_t or NULL (legacy default stream); the call returns
 *          without waiting for the GPU
 * Nothing is allocated: the partial sums live in one fixed 128 KiB device array
 * per GPU, held until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress); make that first call
 * before capturing a stream.  The address is kept for the life of the process:
 * it does not survive cudaDeviceReset (or any new primary context) on that
 * device, after which this call must not be used.  Calls that overlap on the
 * GPU share the array and race; the result is deterministic for a given n. */
int oci_diff_norm_noalloc(const double *a, const double *b, int64_t n, double *e_out, void *stream);

/* Facts of the setup of a single-slab handle (see oci_info). */
int oci_get_info(const oci_handle *h, oci_info *info);

/* Release the handle and its device memory.  NULL is accepted. */
void oci_destroy(oci_handle *h);

/* Message of the last failure on the calling thread ("" if none). */
const char *oci_last_error(void);

/* Krylov acceleration of the FP64 step (beyond the paper, which names Krylov
 * methods as a route to faster convergence, Sec. 4).  One OCI sweep is the
 * affine map F(x) = T x + b (T = A^{-1} B, Eq. oci); with OCI_ACCEL_GMRES each
 * oci_step solves the same fixed point, (I - T) x = b, by restarted GMRES(restart)
 * from the step's initial iterate, one sweep per Krylov vector, and stops when
 * ||F(x) - x||_2 (the e one OCI sweep would make, Sec. 2.1) < tol *
 * residual_factor; it then commits F(x).  oci_stats.iters counts the sweeps,
 * e_last is that residual, rho_e_last is 0.  Needs the FP64 structured solver
 * in Jacobi order; restart in [1, 32]; residual_factor in (0, 1] (0.05 suits
 * contraction rates up to ~0.95: the error is at most the residual / (1 - rho)).
 * Device storage (restart + 3 vectors of the state's size) is allocated at the
 * first accelerated step.  OCI_ACCEL_NONE restores plain OCI. */
enum { OCI_ACCEL_NONE = 0, OCI_ACCEL_GMRES = 1 };
int oci_set_acceleration(oci_handle *h, int32_t accel, int32_t restart, double residual_factor);

/* Fourier (von Neumann) analysis of the iterations (Sec. 2.3), batched on the
 * GPU.  Model problem: infinite homogeneous medium, one group, Sigma_t = v = 1,
 * so case i has cell optical thickness delta[i] (= dx), mean free time tau[i]
 * (= dt; +inf: steady state) and scattering ratio c[i] (= Sigma_s).
 * rho[i] = max over theta_k = 2 pi k / (n_theta - 1), k = 0 .. n_theta-1 (theta
 * = 0 alone if n_theta = 1), of the spectral radius of the iteration operator of
 * a mode e^{i theta j}:
 *   OCI_FOURIER_OCI:   T = (L_c - S)^{-1} B(theta)   (one-cell inversion)
 *   OCI_FOURIER_SI:    T = (L_c - B(theta))^{-1} S   (source iteration)
 *   OCI_FOURIER_MARCH: the time-march amplification of Sec. 2.2 (Eqs. eig1-4,
 *                      K+ and K-), psi_{k+1/2} = K psi_{k-1/2}: the largest
 *                      |eigenvalue| of the per-ordinate 2 x 2 matrix
 *                      K = gamma (K+- K+- + (dx/(v dt)) K+- + gamma I)^{-1},
 *                      gamma = (dx/(v dt)) (dx/(2 v dt)), over theta and the N
 *                      ordinates; the model problem has no scattering, so c is
 *                      not read (it may be NULL); tau = +inf gives 0.
 *                      Unconditional stability is rho <= 1 everywhere.
 * with L_c the cell operator (Eq. Aj), S the within-cell scattering (Eq.
 * scatter, column-angle weight) and B(theta) the lagged inflow.  OCI and SI are
 * computed on reduced matrices with the same nonzero spectrum (2N x 2N for OCI,
 * 4 x 4 for SI) as lim ||M^n||^{1/n} with n = 2^30 (normalised repeated
 * squaring, FP64); MARCH from the closed-form eigenvalues of each 2 x 2 K.
 * N even, 2 <= N <= 32; 1 <= n_cases <= 65535.  delta, tau, c: [n_cases], all host or all device;
 * rho: [n_cases], host or device.  stream: cudaStream_t or NULL.  Blocks until
 * the result is written.  Returns OCI_E_INVAL for bad arguments before any
 * device work. */
enum { OCI_FOURIER_OCI = 0, OCI_FOURIER_SI = 1, OCI_FOURIER_MARCH = 2 };
int oci_fourier_rho(int32_t kind, int32_t N, int32_t n_cases, const double *delta, const double *tau,
                    const double *c, int32_t n_theta, double *rho, void *stream);

/* Measured FP64 fused-multiply-add throughput of the current device in
 * FLOP/s (a register-only DFMA loop, CUDA-event timed): the arithmetic
 * roofline of the FP64 path.  Returns a negative status on failure. */
int oci_probe_fp64_peak(double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* OCI_H */
