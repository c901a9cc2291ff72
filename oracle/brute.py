"""Global direct solve of one SCB x MB time step (test infrastructure only).

Every unknown psi_{j,g,m,p} of every cell of the slab is solved at once: the
four balance equations of each (cell, group, angle) are written straight from
Eqs. scb-mb-a..d of the paper with the midpoint closure (average of the two
corners) and the upstream edge closure, and the incident fluxes at x = 0 and
x = X enter as known edge values.  Nothing is lagged and nothing is iterated;
the dense global matrix is solved by numpy.linalg.solve.

This deliberately does NOT use the within-cell operator L_c of Eq. Aj, the
right-hand side of Eq. rhs_sg or the scattering matrix of Eq. scatter: it is the
plain definition those are derived from, so agreement with the converged OCI
and SI iterations pins all three.
"""
from __future__ import annotations

import numpy as np


def _gl(N):
    return np.polynomial.legendre.leggauss(N)


def solve_step(prob, psi_prev, inc_left=None, inc_right=None):
    """Exact discrete solution Psi[J][G][N][4] of one step from psi_prev[J][G][N][2]."""
    P = prob
    J, N, G = P.J, P.N, P.G
    mu, w = _gl(N)
    inc_left = P.inc_left if inc_left is None else inc_left
    inc_right = P.inc_right if inc_right is None else inc_right
    n = J * G * N * 4

    def ix(j, g, m, p):
        return ((j * G + g) * N + m) * 4 + p

    M = np.zeros((n, n))
    rhs = np.zeros(n)

    def edge(row, coef, j_edge_left_cell, g, m, level):
        """Add coef * psi at edge (j_edge_left_cell + 1/2) for time level
        level (0 = average k, 1 = edge k+1/2) to the equation `row`."""
        jl = j_edge_left_cell          # cell on the left of the edge (-1 at x = 0)
        jr = j_edge_left_cell + 1      # cell on the right of the edge (J at x = X)
        if mu[m] > 0:                  # upstream is the left cell's R corner
            if jl < 0:
                val = 0.0 if inc_left is None else inc_left[g, m, level]
                rhs[row] -= coef * val
            else:
                M[row, ix(jl, g, m, 1 + 2 * level)] += coef
        else:                          # upstream is the right cell's L corner
            if jr >= J:
                val = 0.0 if inc_right is None else inc_right[g, m, level]
                rhs[row] -= coef * val
            else:
                M[row, ix(jr, g, m, 0 + 2 * level)] += coef

    for j in range(J):
        dx = P.dx[j]
        mt = P.mat[j]
        for g in range(G):
            sig = P.sigma_t[mt, g]
            v = P.v[g]
            dt = P.dt
            for m in range(N):
                um = mu[m]
                kL, kR, hL, hR = (ix(j, g, m, p) for p in range(4))
                pL, pR = psi_prev[j, g, m, 0], psi_prev[j, g, m, 1]
                rows = (kL, kR, hL, hR)
                # --- Eq. scb-mb-a (time average, left corner)
                r = rows[0]
                M[r, hL] += dx / 2 / v / dt
                rhs[r] += dx / 2 / v / dt * pL
                M[r, kL] += um / 2
                M[r, kR] += um / 2
                edge(r, -um, j - 1, g, m, 0)
                M[r, kL] += dx / 2 * sig
                # --- Eq. scb-mb-b (time average, right corner)
                r = rows[1]
                M[r, hR] += dx / 2 / v / dt
                rhs[r] += dx / 2 / v / dt * pR
                edge(r, um, j, g, m, 0)
                M[r, kL] -= um / 2
                M[r, kR] -= um / 2
                M[r, kR] += dx / 2 * sig
                # --- Eq. scb-mb-c (time edge, left corner)
                r = rows[2]
                M[r, hL] += dx / 2 / v / (dt / 2)
                M[r, kL] -= dx / 2 / v / (dt / 2)
                M[r, hL] += um / 2
                M[r, hR] += um / 2
                edge(r, -um, j - 1, g, m, 1)
                M[r, hL] += dx / 2 * sig
                # --- Eq. scb-mb-d (time edge, right corner)
                r = rows[3]
                M[r, hR] += dx / 2 / v / (dt / 2)
                M[r, kR] -= dx / 2 / v / (dt / 2)
                edge(r, um, j, g, m, 1)
                M[r, hL] -= um / 2
                M[r, hR] -= um / 2
                M[r, hR] += dx / 2 * sig
                # --- right-hand sides: (dx/2)(1/2)(sum_g' Sigma_s,g'->g sum_n w_n psi_n + Q)
                for p, r in enumerate(rows):
                    for gp in range(G):
                        ss = P.sigma_s[mt, gp, g]
                        for nn in range(N):
                            M[r, ix(j, gp, nn, p)] -= dx / 4 * ss * w[nn]
                    if P.Q is not None:
                        rhs[r] += dx / 4 * P.Q[j, g, p]
    x = np.linalg.solve(M, rhs)
    return x.reshape(J, G, N, 4)


def transient(prob, n_steps, boundary=None):
    """n_steps exact steps; boundary(k) -> (inc_left, inc_right) per step if given.
    Returns the list of Psi per step."""
    P = prob
    psi_prev = np.zeros((P.J, P.G, P.N, 2)) if P.psi_init is None else P.psi_init.copy()
    out = []
    for k in range(n_steps):
        il, ir = boundary(k) if boundary else (None, None)
        Psi = solve_step(P, psi_prev, il, ir)
        out.append(Psi)
        psi_prev = Psi[..., 2:4].copy()
    return out
