/*
 * oci_oracle.c -- plain, slow, FP64 CPU oracle for one-cell inversion (OCI) and
 * source iteration (SI) on the simple-corner-balance (SCB) x multiple-balance (MB)
 * discretisation of time-dependent multigroup slab S_N transport
 * (arXiv 2503.00264, Morgan, Variansyah, Palmer, Niemeyer).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the tests, the package smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator with
 * the CUDA path.
 *
 * Every routine follows the paper's definitions literally: the dense per-cell
 * matrix A_j is assembled element by element (Eqs. Aja/Aj, Eq. scatter, Eq.
 * fullOCIlhs), factored by textbook LU with partial pivoting, and the right-hand
 * side is built from Eq. rhs_sg with the inflow lagged one iteration (Eq. oci).
 * No blocking, fusion or algebraic shortcut is applied.
 *
 * Readings taken where the paper is garbled or silent (each is listed in the
 * design notes of the repository):
 *   R1  scattering matrix (Eq. scatter): S[(g,m,p),(g',n,p')] =
 *       delta_{pp'} * dx/4 * Sigma_s,g'->g * w_n  (weight of the COLUMN angle),
 *       which is what the right-hand side (dx/2)(1/2) Sigma_s sum_n w_n psi_n of
 *       Eqs. scb-mb-a..d gives.
 *   R2  Eq. Aj: every Sigma is the group total cross section Sigma_t,g of the
 *       cell's material, v is v_g.
 *   R3  Q[j][g][p] is the isotropic total emission per corner/time level
 *       (p = kL,kR,hL,hR); the angular source is Q/2.
 *   R4  incident fluxes: inc[g][m][0] is the time-average value over the step,
 *       inc[g][m][1] the value at the step's end edge t_{k+1/2}.
 *   R5  stop rule of Sec. 2.1 / Algorithm 2: e_l = ||Psi^{l+1}-Psi^l||_2;
 *       converged if e_l == 0, else for l >= 1 with rho_e = e_l/e_{l-1},
 *       converged if e_l < tol*(1-rho_e); not converged after max_iter sweeps
 *       -> status ORC_NOCONV and the step is not committed.
 *   R6  SI group coupling (Eq. app:si_update is dimensionally garbled): Jacobi
 *       over groups -- the full scattering source of every group is built from
 *       the lagged scalar flux phi^(l).
 *
 * Layouts (row-major, C order):
 *   Psi      [J][G][N][4]   p = 0 kL, 1 kR, 2 hL, 3 hR  (k: time average,
 *                                                          h: time edge k+1/2)
 *   psi_prev [J][G][N][2]   psi_{k-1/2} at corners L,R
 *   phi      [J][G][4]
 *   Q        [J][G][4]
 *   sigma_t  [n_mat][G]; sigma_s [n_mat][G][G] with sigma_s[m][gp][g] = Sigma_s,gp->g
 *   inc_left/inc_right [G][N][2]
 *   unknown index inside a cell: idx(g,m,p) = (g*N + m)*4 + p   (Eq. x_vec)
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVAL (-1)
#define ORC_NOMEM (-2)
#define ORC_NOCONV (-4)
#define ORC_SINGULAR (-5)

typedef struct {
  int32_t J, N, G, n_mat;
  const double *dx;        /* [J]            */
  const int32_t *mat;      /* [J]            */
  const double *sigma_t;   /* [n_mat][G]     */
  const double *sigma_s;   /* [n_mat][G][G]  */
  const double *v;         /* [G]            */
  const double *Q;         /* [J][G][4] or NULL */
  double dt;
  const double *inc_left;  /* [G][N][2] or NULL */
  const double *inc_right; /* [G][N][2] or NULL */
  /* Optional factor sharing.  Cells whose (material, dx) are equal have
   * bit-identical A_j (A_j depends on nothing else), so their LU factors are
   * identical too; with slot_of_cell != NULL the factors are stored once per
   * slot: slot_of_cell[j] in [0, n_slots) names the factor of cell j and
   * slot_first_cell[s] the cell that slot s is factored from.  NULL: one
   * factor per cell (slot = j).  Results are the same bits either way.        */
  int32_t n_slots;
  const int32_t *slot_of_cell;    /* [J] or NULL       */
  const int32_t *slot_first_cell; /* [n_slots] or NULL */
} orc_problem;

static size_t lu_slot(const orc_problem *p, int j) {
  return p->slot_of_cell ? (size_t)p->slot_of_cell[j] : (size_t)j;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre quadrature on [-1,1] (the S_N set used throughout the paper,
 * Sec. 1 footnote).  Newton's method on the Legendre polynomial P_N evaluated by
 * its three-term recurrence; ascending mu.                                      */
int orc_gauss_legendre(int32_t N, double *mu, double *w) {
  if (N < 1) return ORC_INVAL;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < N; i++) {
    /* initial guess for the i-th largest root */
    double x = cos(pi * (i + 0.75) / (N + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; it++) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= N; k++) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pN = (N == 1) ? x : p1;
      double pNm1 = (N == 1) ? 1.0 : p0;
      dp = N * (x * pN - pNm1) / (x * x - 1.0);
      double dxn = pN / dp;
      x -= dxn;
      if (fabs(dxn) < 1e-16) break;
    }
    /* recompute derivative at the converged root */
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= N; k++) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pN = (N == 1) ? x : p1;
      double pNm1 = (N == 1) ? 1.0 : p0;
      dp = N * (x * pN - pNm1) / (x * x - 1.0);
    }
    /* i-th largest root goes to position N-1-i (ascending order) */
    mu[N - 1 - i] = x;
    w[N - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
static size_t idx_cell(const orc_problem *p, int g, int m, int q) {
  return ((size_t)g * p->N + m) * 4 + q;
}

/* Dense A_j of order 4NG (row-major), Eqs. Aja, Aj, scatter, fullOCIlhs.     */
int orc_cell_matrix(const orc_problem *p, const double *mu, const double *w, int32_t j, double *A) {
  const int N = p->N, G = p->G;
  const size_t n = (size_t)4 * N * G;
  const double dxj = p->dx[j];
  const int mt = p->mat[j];
  memset(A, 0, n * n * sizeof(double));
  for (int g = 0; g < G; g++) {
    const double sig = p->sigma_t[(size_t)mt * G + g];
    const double alpha = dxj / (p->v[g] * p->dt); /* dx/(v dt) */
    for (int m = 0; m < N; m++) {
      const double a = (fabs(mu[m]) + dxj * sig) / 2.0;
      const size_t r0 = idx_cell(p, g, m, 0);
      double L[4][4] = {
          {a, mu[m] / 2.0, alpha / 2.0, 0.0},
          {-mu[m] / 2.0, a, 0.0, alpha / 2.0},
          {-alpha, 0.0, alpha + a, mu[m] / 2.0},
          {0.0, -alpha, -mu[m] / 2.0, alpha + a},
      };
      for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) A[(r0 + r) * n + (r0 + c)] += L[r][c];
    }
  }
  /* within-cell scattering, all groups: row (g,m,q), column (gp,nn,q) */
  for (int g = 0; g < G; g++)
    for (int m = 0; m < N; m++)
      for (int q = 0; q < 4; q++) {
        const size_t r = idx_cell(p, g, m, q);
        for (int gp = 0; gp < G; gp++) {
          const double ss = p->sigma_s[((size_t)mt * G + gp) * G + g]; /* gp -> g */
          for (int nn = 0; nn < N; nn++) {
            const size_t c = idx_cell(p, gp, nn, q);
            A[r * n + c] -= dxj / 4.0 * ss * w[nn];
          }
        }
      }
  return ORC_OK;
}

/* Textbook LU with partial pivoting (first max-|.| row on ties).             */
int orc_lu_factor(int32_t n, double *A, int32_t *piv) {
  for (int k = 0; k < n; k++) {
    int pr = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int r = k + 1; r < n; r++) {
      double v = fabs(A[(size_t)r * n + k]);
      if (v > best) {
        best = v;
        pr = r;
      }
    }
    piv[k] = pr;
    if (best == 0.0) return ORC_SINGULAR;
    if (pr != k)
      for (int c = 0; c < n; c++) {
        double t = A[(size_t)k * n + c];
        A[(size_t)k * n + c] = A[(size_t)pr * n + c];
        A[(size_t)pr * n + c] = t;
      }
    for (int r = k + 1; r < n; r++) {
      double l = A[(size_t)r * n + k] / A[(size_t)k * n + k];
      A[(size_t)r * n + k] = l;
      for (int c = k + 1; c < n; c++) A[(size_t)r * n + c] -= l * A[(size_t)k * n + c];
    }
  }
  return ORC_OK;
}

void orc_lu_solve(int32_t n, const double *LU, const int32_t *piv, double *b) {
  for (int k = 0; k < n; k++) {
    int pr = piv[k];
    if (pr != k) {
      double t = b[k];
      b[k] = b[pr];
      b[pr] = t;
    }
  }
  for (int r = 0; r < n; r++) {
    double s = b[r];
    for (int c = 0; c < r; c++) s -= LU[(size_t)r * n + c] * b[c];
    b[r] = s;
  }
  for (int r = n - 1; r >= 0; r--) {
    double s = b[r];
    for (int c = r + 1; c < n; c++) s -= LU[(size_t)r * n + c] * b[c];
    b[r] = s / LU[(size_t)r * n + r];
  }
}

/* Factor every cell's A_j (the paper's gesv on the first iteration, done once);
 * with factor sharing, once per slot from its first cell.                       */
int orc_factor_all(const orc_problem *p, const double *mu, const double *w, double *LU, int32_t *piv) {
  const size_t n = (size_t)4 * p->N * p->G;
  const int nf = p->slot_of_cell ? p->n_slots : p->J;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int s = 0; s < nf; s++) {
    const int j = p->slot_of_cell ? p->slot_first_cell[s] : s;
    double *A = LU + (size_t)s * n * n;
    orc_cell_matrix(p, mu, w, j, A);
    if (orc_lu_factor((int32_t)n, A, piv + (size_t)s * n) != ORC_OK) bad = 1;
  }
  return bad ? ORC_SINGULAR : ORC_OK;
}

/* Right-hand side b_j, Eq. rhs_sg extended to groups (Eq. fullOCIrhs), with the
 * incident angular fluxes lagged from the previous iterate Psi_l.                */
void orc_rhs(const orc_problem *p, const double *mu, int32_t j, const double *psi_prev,
             const double *Psi_l, double *b) {
  const int J = p->J, N = p->N, G = p->G;
  const double dxj = p->dx[j];
  for (int g = 0; g < G; g++) {
    const double alpha = dxj / (p->v[g] * p->dt);
    const double *q = p->Q ? p->Q + ((size_t)j * G + g) * 4 : NULL;
    for (int m = 0; m < N; m++) {
      double *bb = b + idx_cell(p, g, m, 0);
      const double *pp = psi_prev + (((size_t)j * G + g) * N + m) * 2;
      for (int r = 0; r < 4; r++) bb[r] = q ? dxj / 4.0 * q[r] : 0.0;
      bb[0] += alpha / 2.0 * pp[0];
      bb[1] += alpha / 2.0 * pp[1];
      if (mu[m] > 0) {
        double uk, uh;
        if (j > 0) {
          const double *up = Psi_l + (((size_t)(j - 1) * G + g) * N + m) * 4;
          uk = up[1];
          uh = up[3];
        } else {
          uk = p->inc_left ? p->inc_left[((size_t)g * N + m) * 2 + 0] : 0.0;
          uh = p->inc_left ? p->inc_left[((size_t)g * N + m) * 2 + 1] : 0.0;
        }
        bb[0] += mu[m] * uk;
        bb[2] += mu[m] * uh;
      } else {
        double uk, uh;
        if (j < J - 1) {
          const double *up = Psi_l + (((size_t)(j + 1) * G + g) * N + m) * 4;
          uk = up[0];
          uh = up[2];
        } else {
          uk = p->inc_right ? p->inc_right[((size_t)g * N + m) * 2 + 0] : 0.0;
          uh = p->inc_right ? p->inc_right[((size_t)g * N + m) * 2 + 1] : 0.0;
        }
        bb[1] -= mu[m] * uk;
        bb[3] -= mu[m] * uh;
      }
    }
  }
}

/* One OCI sweep (block Jacobi over cells, Eq. oci): Psi_new_j = A_j^{-1} b_j(Psi_l)
 * for every cell; returns e = ||Psi_new - Psi_l||_2 summed in cell order.       */
double orc_oci_sweep(const orc_problem *p, const double *mu, const double *LU, const int32_t *piv,
                     const double *psi_prev, const double *Psi_l, double *Psi_new) {
  const size_t n = (size_t)4 * p->N * p->G;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < p->J; j++) {
    double *b = Psi_new + (size_t)j * n;
    orc_rhs(p, mu, j, psi_prev, Psi_l, b);
    orc_lu_solve((int32_t)n, LU + lu_slot(p, j) * n * n, piv + lu_slot(p, j) * n, b);
  }
  double s = 0.0;
  for (size_t i = 0; i < (size_t)p->J * n; i++) {
    double d = Psi_new[i] - Psi_l[i];
    s += d * d;
  }
  return sqrt(s);
}

/* One red-black OCI sweep (cell-wise block Gauss-Seidel in red-black order,
 * Sec. 1 of the paper names it beside block Jacobi): first every even cell is
 * solved with the inflow of the current (old) odd cells, then every odd cell
 * with the inflow of the just-updated even cells.  Psi_new starts as a copy of
 * Psi_l and is updated in place; returns ||Psi_new - Psi_l||_2.              */
double orc_rb_sweep(const orc_problem *p, const double *mu, const double *LU, const int32_t *piv,
                    const double *psi_prev, const double *Psi_l, double *Psi_new) {
  const size_t n = (size_t)4 * p->N * p->G;
  memcpy(Psi_new, Psi_l, (size_t)p->J * n * sizeof(double));
  double *b = (double *)malloc(n * sizeof(double));
  for (int color = 0; color < 2; color++)
    for (int j = color; j < p->J; j += 2) {
      orc_rhs(p, mu, j, psi_prev, Psi_new, b);
      orc_lu_solve((int32_t)n, LU + lu_slot(p, j) * n * n, piv + lu_slot(p, j) * n, b);
      memcpy(Psi_new + (size_t)j * n, b, n * sizeof(double));
    }
  free(b);
  double s = 0.0;
  for (size_t i = 0; i < (size_t)p->J * n; i++) {
    double d = Psi_new[i] - Psi_l[i];
    s += d * d;
  }
  return sqrt(s);
}

/* Per-cell solve for a list of cells only (sampled checks at full size).      */
int orc_oci_cells(const orc_problem *p, const double *mu, const double *w, const double *psi_prev,
                  const double *Psi_l, int32_t ncells, const int32_t *cells, double *out) {
  const size_t n = (size_t)4 * p->N * p->G;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int i = 0; i < ncells; i++) {
    double *A = (double *)malloc(n * n * sizeof(double));
    int32_t *pv = (int32_t *)malloc(n * sizeof(int32_t));
    if (!A || !pv) {
      bad = 1;
    } else {
      const int j = cells[i];
      orc_cell_matrix(p, mu, w, j, A);
      if (orc_lu_factor((int32_t)n, A, pv) != ORC_OK) bad = 1;
      double *b = out + (size_t)i * n;
      orc_rhs(p, mu, j, psi_prev, Psi_l, b);
      orc_lu_solve((int32_t)n, A, pv, b);
    }
    free(A);
    free(pv);
  }
  return bad ? ORC_SINGULAR : ORC_OK;
}

/* Scalar flux phi_{j,g,p} = sum_m w_m Psi_{j,g,m,p} (Eq. app:si_sf).           */
void orc_scalar_flux(const orc_problem *p, const double *w, const double *Psi, double *phi) {
  const int N = p->N, G = p->G;
  for (int j = 0; j < p->J; j++)
    for (int g = 0; g < G; g++)
      for (int q = 0; q < 4; q++) {
        double s = 0.0;
        for (int m = 0; m < N; m++) s += w[m] * Psi[(((size_t)j * G + g) * N + m) * 4 + q];
        phi[((size_t)j * G + g) * 4 + q] = s;
      }
}

/* One SI sweep (Algorithm 1, App. A, Eqs. app:si_sys, app:si_rhs): for every
 * (g,m), march through the cells in the direction of flight solving the 4x4
 * L_{c,j,g,m} psi = d with the current sweep's upstream edge and the scattering
 * source from the lagged scalar flux phi_l (reading R6).  Writes Psi_new and
 * phi_new; returns ||phi_new - phi_l||_2.                                      */
double orc_si_sweep(const orc_problem *p, const double *mu, const double *w, const double *psi_prev,
                    const double *phi_l, double *Psi_new, double *phi_new) {
  const int J = p->J, N = p->N, G = p->G;
#pragma omp parallel for schedule(dynamic, 1)
  for (int gm = 0; gm < G * N; gm++) {
    const int g = gm / N, m = gm % N;
    double uk, uh;
    const double *inc = mu[m] > 0 ? p->inc_left : p->inc_right;
    uk = inc ? inc[((size_t)g * N + m) * 2 + 0] : 0.0;
    uh = inc ? inc[((size_t)g * N + m) * 2 + 1] : 0.0;
    for (int s = 0; s < J; s++) {
      const int j = mu[m] > 0 ? s : J - 1 - s;
      const double dxj = p->dx[j];
      const int mt = p->mat[j];
      const double sig = p->sigma_t[(size_t)mt * G + g];
      const double alpha = dxj / (p->v[g] * p->dt);
      const double a = (fabs(mu[m]) + dxj * sig) / 2.0;
      double L[16] = {a,      mu[m] / 2.0, alpha / 2.0, 0.0,          -mu[m] / 2.0, a,
                      0.0,    alpha / 2.0, -alpha,      0.0,          alpha + a,    mu[m] / 2.0,
                      0.0,    -alpha,      -mu[m] / 2.0, alpha + a};
      int32_t pv[4];
      double d[4];
      const double *pp = psi_prev + (((size_t)j * G + g) * N + m) * 2;
      for (int q = 0; q < 4; q++) {
        double src = p->Q ? p->Q[((size_t)j * G + g) * 4 + q] : 0.0;
        for (int gp = 0; gp < G; gp++)
          src += p->sigma_s[((size_t)mt * G + gp) * G + g] * phi_l[((size_t)j * G + gp) * 4 + q];
        d[q] = dxj / 4.0 * src;
      }
      d[0] += alpha / 2.0 * pp[0];
      d[1] += alpha / 2.0 * pp[1];
      if (mu[m] > 0) {
        d[0] += mu[m] * uk;
        d[2] += mu[m] * uh;
      } else {
        d[1] -= mu[m] * uk;
        d[3] -= mu[m] * uh;
      }
      orc_lu_factor(4, L, pv);
      orc_lu_solve(4, L, pv, d);
      double *out = Psi_new + (((size_t)j * G + g) * N + m) * 4;
      for (int q = 0; q < 4; q++) out[q] = d[q];
      if (mu[m] > 0) {
        uk = d[1];
        uh = d[3];
      } else {
        uk = d[0];
        uh = d[2];
      }
    }
  }
  orc_scalar_flux(p, w, Psi_new, phi_new);
  double s = 0.0;
  for (size_t i = 0; i < (size_t)J * G * 4; i++) {
    double d = phi_new[i] - phi_l[i];
    s += d * d;
  }
  return sqrt(s);
}

/* Particle balance tallies of one committed step, per group.
 * Summing Eqs. scb-mb-a + scb-mb-b (time-average balance, b = 0) and
 * scb-mb-c + scb-mb-d (time-edge balance, b = 1) over corners, angles (weights
 * w_m) and cells gives, for each group g,
 *   time + leak + collision - scatter_in - source = 0,
 * exactly for the discrete solution and to O(e) for an OCI iterate.
 * bal[g][b][0..4] = {time, leak, collision, scatter_in, source}.               */
void orc_balance(const orc_problem *p, const double *mu, const double *w, const double *psi_prev,
                 const double *Psi, double *bal) {
  const int J = p->J, N = p->N, G = p->G;
  double *phi = (double *)calloc((size_t)J * G * 4, sizeof(double));
  orc_scalar_flux(p, w, Psi, phi);
  for (int g = 0; g < G; g++) {
    double tA = 0, cA = 0, sA = 0, qA = 0, tE = 0, cE = 0, sE = 0, qE = 0;
    for (int j = 0; j < J; j++) {
      const double dxj = p->dx[j];
      const int mt = p->mat[j];
      const double sig = p->sigma_t[(size_t)mt * G + g];
      const double rate = dxj / (p->v[g] * p->dt);
      const double *ph = phi + ((size_t)j * G + g) * 4;
      double phiprev[2] = {0, 0};
      for (int m = 0; m < N; m++) {
        phiprev[0] += w[m] * psi_prev[(((size_t)j * G + g) * N + m) * 2 + 0];
        phiprev[1] += w[m] * psi_prev[(((size_t)j * G + g) * N + m) * 2 + 1];
      }
      tA += rate / 2.0 * ((ph[2] - phiprev[0]) + (ph[3] - phiprev[1]));
      tE += rate * ((ph[2] - ph[0]) + (ph[3] - ph[1]));
      cA += dxj / 2.0 * sig * (ph[0] + ph[1]);
      cE += dxj / 2.0 * sig * (ph[2] + ph[3]);
      for (int gp = 0; gp < G; gp++) {
        const double ss = p->sigma_s[((size_t)mt * G + gp) * G + g];
        const double *pg = phi + ((size_t)j * G + gp) * 4;
        sA += dxj / 2.0 * ss * (pg[0] + pg[1]);
        sE += dxj / 2.0 * ss * (pg[2] + pg[3]);
      }
      if (p->Q) {
        const double *q = p->Q + ((size_t)j * G + g) * 4;
        qA += dxj / 2.0 * (q[0] + q[1]);
        qE += dxj / 2.0 * (q[2] + q[3]);
      }
    }
    /* leakage: sum_m w_m mu_m (psi at right edge - psi at left edge), upstream */
    double lA = 0, lE = 0;
    for (int m = 0; m < N; m++) {
      double rk, rh, lk, lh;
      if (mu[m] > 0) {
        const double *c = Psi + (((size_t)(J - 1) * G + g) * N + m) * 4;
        rk = c[1];
        rh = c[3];
        lk = p->inc_left ? p->inc_left[((size_t)g * N + m) * 2 + 0] : 0.0;
        lh = p->inc_left ? p->inc_left[((size_t)g * N + m) * 2 + 1] : 0.0;
      } else {
        const double *c = Psi + (((size_t)0 * G + g) * N + m) * 4;
        lk = c[0];
        lh = c[2];
        rk = p->inc_right ? p->inc_right[((size_t)g * N + m) * 2 + 0] : 0.0;
        rh = p->inc_right ? p->inc_right[((size_t)g * N + m) * 2 + 1] : 0.0;
      }
      lA += w[m] * mu[m] * (rk - lk);
      lE += w[m] * mu[m] * (rh - lh);
    }
    double *bg = bal + (size_t)g * 10;
    bg[0] = tA; bg[1] = lA; bg[2] = cA; bg[3] = sA; bg[4] = qA;
    bg[5] = tE; bg[6] = lE; bg[7] = cE; bg[8] = sE; bg[9] = qE;
  }
  free(phi);
}

/* Stop rule (reading R5).  Returns 1 when converged after sweep l.            */
static int stop_rule(int l, double e, double e_prev, double tol, double *rho) {
  if (e == 0.0) {
    *rho = 0.0;
    return 1;
  }
  if (l >= 1) {
    *rho = e / e_prev;
    return e < tol * (1.0 - *rho);
  }
  *rho = 0.0;
  return 0;
}

/* One time step by OCI (method 0), SI (method 1) or red-black OCI (method 2).
 *  Psi_io   in: the initial iterate Psi^(0) (the caller applies its guess policy)
 *           out: the last iterate (the converged Psi_k on success)
 *  psi_prev in: psi_{k-1/2}; out on success: psi_{k+1/2} = (Psi hL, Psi hR)
 *  phi_out  [J][G][4] scalar flux of the committed step (may be NULL)
 *  bal_out  [G][2][5] balance tallies of the committed step (may be NULL)
 *  stats    {iters, e_last, rho_last}
 *  e_hist   [max_iter] per-sweep e (may be NULL)
 *  LU/piv   from orc_factor_all (OCI only; may be NULL for SI)
 * Returns ORC_OK, or ORC_NOCONV (nothing committed: psi_prev untouched).       */
int orc_step(const orc_problem *p, int32_t method, double tol, int32_t max_iter, const double *LU,
             const int32_t *piv, double *psi_prev, double *Psi_io, double *phi_out, double *bal_out,
             double *stats, double *e_hist) {
  const int J = p->J, N = p->N, G = p->G;
  const size_t nPsi = (size_t)J * G * N * 4, nphi = (size_t)J * G * 4;
  double mu[1024], w[1024];
  if (N > 1024 || max_iter < 1) return ORC_INVAL;
  orc_gauss_legendre(N, mu, w);
  double *Psi_a = (double *)malloc(nPsi * sizeof(double));
  double *phi_a = (double *)malloc(nphi * sizeof(double));
  double *phi_b = (double *)malloc(nphi * sizeof(double));
  if (!Psi_a || !phi_a || !phi_b) {
    free(Psi_a); free(phi_a); free(phi_b);
    return ORC_NOMEM;
  }
  double e = 0, e_prev = 0, rho = 0;
  int conv = 0, l = 0;
  if (method == 1) orc_scalar_flux(p, w, Psi_io, phi_a);
  for (l = 0; l < max_iter; l++) {
    if (method == 0 || method == 2) {
      e = method == 0 ? orc_oci_sweep(p, mu, LU, piv, psi_prev, Psi_io, Psi_a)
                      : orc_rb_sweep(p, mu, LU, piv, psi_prev, Psi_io, Psi_a);
      memcpy(Psi_io, Psi_a, nPsi * sizeof(double));
    } else {
      e = orc_si_sweep(p, mu, w, psi_prev, phi_a, Psi_io, phi_b);
      memcpy(phi_a, phi_b, nphi * sizeof(double));
    }
    if (e_hist) e_hist[l] = e;
    conv = stop_rule(l, e, e_prev, tol, &rho);
    e_prev = e;
    if (conv) break;
  }
  int iters = conv ? l + 1 : max_iter;
  if (stats) {
    stats[0] = iters;
    stats[1] = e;
    stats[2] = rho;
  }
  if (conv) {
    if (bal_out) orc_balance(p, mu, w, psi_prev, Psi_io, bal_out);
    if (phi_out) orc_scalar_flux(p, w, Psi_io, phi_out);
    for (int j = 0; j < J; j++)
      for (int g = 0; g < G; g++)
        for (int m = 0; m < N; m++) {
          const double *c = Psi_io + (((size_t)j * G + g) * N + m) * 4;
          double *pp = psi_prev + (((size_t)j * G + g) * N + m) * 2;
          pp[0] = c[2];
          pp[1] = c[3];
        }
  }
  free(Psi_a); free(phi_a); free(phi_b);
  return conv ? ORC_OK : ORC_NOCONV;
}

/* Exactly n sweeps from Psi_io with no stop test and no commit.               */
int orc_iterate(const orc_problem *p, int32_t method, int32_t n, const double *LU, const int32_t *piv,
                const double *psi_prev, double *Psi_io, double *e_hist) {
  const int J = p->J, N = p->N, G = p->G;
  const size_t nPsi = (size_t)J * G * N * 4, nphi = (size_t)J * G * 4;
  double mu[1024], w[1024];
  if (N > 1024 || n < 0) return ORC_INVAL;
  orc_gauss_legendre(N, mu, w);
  double *Psi_a = (double *)malloc(nPsi * sizeof(double));
  double *phi_a = (double *)malloc(nphi * sizeof(double));
  double *phi_b = (double *)malloc(nphi * sizeof(double));
  if (!Psi_a || !phi_a || !phi_b) {
    free(Psi_a); free(phi_a); free(phi_b);
    return ORC_NOMEM;
  }
  if (method == 1) orc_scalar_flux(p, w, Psi_io, phi_a);
  for (int l = 0; l < n; l++) {
    double e;
    if (method == 0 || method == 2) {
      e = method == 0 ? orc_oci_sweep(p, mu, LU, piv, psi_prev, Psi_io, Psi_a)
                      : orc_rb_sweep(p, mu, LU, piv, psi_prev, Psi_io, Psi_a);
      memcpy(Psi_io, Psi_a, nPsi * sizeof(double));
    } else {
      e = orc_si_sweep(p, mu, w, psi_prev, phi_a, Psi_io, phi_b);
      memcpy(phi_a, phi_b, nphi * sizeof(double));
    }
    if (e_hist) e_hist[l] = e;
  }
  free(Psi_a); free(phi_a); free(phi_b);
  return ORC_OK;
}

/* Thread count of the OpenMP loops above (used only to time the oracle on one
 * core and on all cores; results do not depend on it).                        */
void orc_set_threads(int32_t n) { omp_set_num_threads(n > 0 ? n : 1); }
int32_t orc_get_threads(void) { return omp_get_max_threads(); }
