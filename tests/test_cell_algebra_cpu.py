"""CPU check of the algebra the FP64 sweep kernels use for the exact cell solve,
restated here in numpy from the balance equations, against the oracle's own
dense cell matrix A_j and right-hand side b_j (Eqs. Aj, scatter, fullOCIlhs,
rhs_sg): for random cells and lagged iterates both forms give A_j^{-1} b_j to
rounding.

  staged form:     t_m = tc_m + C_in,m u_m,  y = sum_m w_m t_m,  s = M' y,
                   Psi_m = t_m + L_m^{-1} s
  register form:   y = y_c + sum_m (w_m C_in,m) u_m,  y_c = sum_m w_m tc_m,
                   s = M' y,  Psi_m = tc_m + L_m^{-1} (s + |mu_m| u_m in the
                   inflow rows)

with tc_m = L_m^{-1} c_m (c: the per-step constant), C_in,m = |mu_m| times the
two columns of L_m^{-1} that the inflow feeds (rows 0, 2 for mu > 0; 1, 3 for
mu < 0), H = blockdiag_g sum_m w_m L_{g,m}^{-1}, K[g][g'] = dx/4 Sigma_s,g'->g,
M' = (I - K H)^{-1} K."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2503_00264_gb300 import workloads as W


def _blocks(p, o, j):
    N, G = p.N, p.G
    mat, dx = int(p.mat[j]), float(p.dx[j])
    Linv = np.zeros((G, N, 4, 4))
    for g in range(G):
        al = dx / (p.v[g] * p.dt)
        for m in range(N):
            mu = o.mu[m]
            a = (abs(mu) + dx * p.sigma_t[mat, g]) / 2.0
            L = np.array([[a, mu / 2, al / 2, 0.0], [-mu / 2, a, 0.0, al / 2],
                          [-al, 0.0, al + a, mu / 2], [0.0, -al, -mu / 2, al + a]])
            Linv[g, m] = np.linalg.inv(L)
    rows = [(0, 2) if o.mu[m] > 0 else (1, 3) for m in range(N)]
    Cin = np.zeros((G, N, 4, 2))
    for g in range(G):
        for m in range(N):
            Cin[g, m] = abs(o.mu[m]) * Linv[g, m][:, list(rows[m])]
    H = np.zeros((4 * G, 4 * G))
    K = np.zeros((4 * G, 4 * G))
    for g in range(G):
        H[4 * g:4 * g + 4, 4 * g:4 * g + 4] = np.einsum("m,mpq->pq", o.w, Linv[g])
        for gp in range(G):
            K[4 * g:4 * g + 4, 4 * gp:4 * gp + 4] = dx / 4 * p.sigma_s[mat, gp, g] * np.eye(4)
    Mp = np.linalg.solve(np.eye(4 * G) - K @ H, K)
    return Linv, Cin, Mp, rows


def _inflow(p, o, j, Psi_l):
    u = np.zeros((p.G, p.N, 2))
    for g in range(p.G):
        for m in range(p.N):
            if o.mu[m] > 0:
                u[g, m] = Psi_l[j - 1, g, m, [1, 3]]
            else:
                u[g, m] = Psi_l[j + 1, g, m, [0, 2]]
    return u


@pytest.mark.parametrize("seed,N,G", [(201, 4, 1), (202, 8, 2), (203, 16, 1), (204, 8, 3), (205, 2, 4)])
def test_staged_and_register_forms_equal_the_dense_solve(seed, N, G):
    p = W.random_slab(seed, 6, N, G)
    o = Oracle(p, factor=False)
    rng = np.random.default_rng(seed)
    for j in (1, 2, 4):  # interior cells: the inflow comes from the lagged iterate
        Psi_l = rng.uniform(0.0, 2.0, size=(p.J, G, N, 4))
        A = o.cell_matrix(j)
        b = o.rhs(j, Psi_l)
        ref = np.linalg.solve(A, b).reshape(G, N, 4)
        c = o.rhs(j, np.zeros_like(Psi_l)).reshape(G, N, 4)  # interior cell: no inflow term
        Linv, Cin, Mp, rows = _blocks(p, o, j)
        u = _inflow(p, o, j, Psi_l)
        tc = np.einsum("gmpq,gmq->gmp", Linv, c)
        # staged form
        t = tc + np.einsum("gmpk,gmk->gmp", Cin, u)
        y = np.einsum("m,gmp->gp", o.w, t).reshape(4 * G)
        s = (Mp @ y).reshape(G, 4)
        psi_staged = t + np.einsum("gmpq,gq->gmp", Linv, s)
        # register form
        yc = np.einsum("m,gmp->gp", o.w, tc)
        y2 = (yc + np.einsum("m,gmpk,gmk->gp", o.w, Cin, u)).reshape(4 * G)
        s2 = (Mp @ y2).reshape(G, 4)
        v = np.repeat(s2[:, None, :], N, axis=1)
        for m in range(N):
            r0, r1 = rows[m]
            v[:, m, r0] += abs(o.mu[m]) * u[:, m, 0]
            v[:, m, r1] += abs(o.mu[m]) * u[:, m, 1]
        psi_reg = tc + np.einsum("gmpq,gmq->gmp", Linv, v)
        scale = np.abs(ref).max()
        assert np.abs(psi_staged - ref).max() < 1e-12 * scale
        assert np.abs(psi_reg - ref).max() < 1e-12 * scale


@pytest.mark.parametrize("seed,N,G", [(211, 4, 1), (212, 8, 2), (213, 16, 3)])
def test_refinement_residual_equals_b_minus_A_psi(seed, N, G):
    """The FP64 residual of the mixed forms' refinement, restated from the
    kernel's row formulas (r = c + s + inflow - L_c Psi with s_g = sum_g'
    dx/4 Sigma_s,g'->g phi_g'), equals b_j - A_j Psi_j from the oracle's dense
    cell matrix for random iterates."""
    p = W.random_slab(seed, 6, N, G)
    o = Oracle(p, factor=False)
    rng = np.random.default_rng(seed)
    for j in (1, 3, 4):
        Psi = rng.uniform(-1.0, 2.0, size=(p.J, G, N, 4))
        ref = o.rhs(j, Psi) - o.cell_matrix(j) @ Psi[j].reshape(-1)
        c = o.rhs(j, np.zeros_like(Psi)).reshape(G, N, 4)
        mat, dx = int(p.mat[j]), float(p.dx[j])
        phi = np.einsum("m,gmp->gp", o.w, Psi[j])
        r = np.zeros((G, N, 4))
        for g in range(G):
            s = sum(dx / 4 * p.sigma_s[mat, gp, g] * phi[gp] for gp in range(G))
            al = dx / (p.v[g] * p.dt)
            for m in range(N):
                mu = o.mu[m]
                a = (abs(mu) + dx * p.sigma_t[mat, g]) / 2
                hm, ha, aa = mu / 2, al / 2, al + a
                v0, v1, v2, v3 = Psi[j, g, m]
                rr = c[g, m] + s
                if mu > 0:
                    rr[0] += mu * Psi[j - 1, g, m, 1]
                    rr[2] += mu * Psi[j - 1, g, m, 3]
                else:
                    rr[1] += -mu * Psi[j + 1, g, m, 0]
                    rr[3] += -mu * Psi[j + 1, g, m, 2]
                rr[0] -= a * v0 + hm * v1 + ha * v2
                rr[1] -= -hm * v0 + a * v1 + ha * v3
                rr[2] -= -al * v0 + aa * v2 + hm * v3
                rr[3] -= -al * v1 - hm * v2 + aa * v3
                r[g, m] = rr
        assert np.abs(r.reshape(-1) - ref).max() < 1e-12 * np.abs(o.rhs(j, Psi)).max()


@pytest.mark.parametrize("seed,J,N,G", [(221, 1, 2, 1), (222, 37, 8, 1), (223, 64, 4, 2), (224, 100, 16, 1)])
def test_si_scan_composition_equals_the_sequential_sweep(seed, J, N, G):
    """The scan form of SI: per (g, m) the outgoing edge of cell j is an affine
    map u_out = T_j u_in + e_j of its incoming edge (T_j = |mu| times the 2x2 block
    of L_j^{-1} from the inflow rows to the outflow corners, e_j the outflow corners
    of L_j^{-1} d_j), the maps compose associatively ((T2, e2) after (T1, e1) =
    (T2 T1, T2 e1 + e2)), and a log-depth inclusive scan of them gives every
    cell's incoming edge.  Restated here in numpy, one SI sweep this way equals
    the oracle's sequential sweep (Algorithm 1)."""
    p = W.random_slab(seed, J, N, G)
    o = Oracle(p, factor=False)
    rng = np.random.default_rng(seed)
    Psi0 = rng.uniform(0.0, 1.0, size=(J, G, N, 4))
    o.Psi[...] = Psi0
    o.iterate(1, method=1)  # one SI sweep from Psi0
    ref = o.Psi.copy()
    phi = np.einsum("m,jgmp->jgp", o.w, Psi0)
    got = np.zeros_like(ref)
    for g in range(G):
        for m in range(N):
            mu = o.mu[m]
            order = list(range(J)) if mu > 0 else list(range(J - 1, -1, -1))
            rin, rout = ([0, 2], [1, 3]) if mu > 0 else ([1, 3], [0, 2])
            inc = p.inc_left if mu > 0 else p.inc_right
            u0 = np.zeros(2) if inc is None else np.array(inc[g, m])
            Li, d, T, e = [], [], [], []
            for j in order:
                mat, dx = int(p.mat[j]), float(p.dx[j])
                al = dx / (p.v[g] * p.dt)
                a = (abs(mu) + dx * p.sigma_t[mat, g]) / 2
                L = np.array([[a, mu / 2, al / 2, 0.0], [-mu / 2, a, 0.0, al / 2],
                              [-al, 0.0, al + a, mu / 2], [0.0, -al, -mu / 2, al + a]])
                src = (0.0 if p.Q is None else p.Q[j, g]) + sum(p.sigma_s[mat, gp, g] * phi[j, gp] for gp in range(G))
                dj = dx / 4 * np.broadcast_to(src, (4,)).astype(float).copy()
                dj[0] += al / 2 * o.psi_prev[j, g, m, 0]
                dj[1] += al / 2 * o.psi_prev[j, g, m, 1]
                inv = np.linalg.inv(L)
                Li.append(inv)
                d.append(dj)
                T.append(abs(mu) * inv[np.ix_(rout, rin)])
                e.append((inv @ dj)[rout])
            # Hillis-Steele inclusive scan of the affine maps
            ST, Se = [t.copy() for t in T], [x.copy() for x in e]
            off = 1
            while off < J:
                nT, ne = [t.copy() for t in ST], [x.copy() for x in Se]
                for i in range(off, J):
                    nT[i] = ST[i] @ ST[i - off]
                    ne[i] = ST[i] @ Se[i - off] + Se[i]
                ST, Se, off = nT, ne, off * 2
            for s, j in enumerate(order):
                uin = u0 if s == 0 else ST[s - 1] @ u0 + Se[s - 1]
                rhs = d[s].copy()
                rhs[rin] += abs(mu) * uin
                got[j, g, m] = Li[s] @ rhs
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("seed,J,N,G", [(231, 9, 4, 1), (232, 12, 8, 2)])
def test_correction_refinement_converges_to_the_global_solve(seed, J, N, G):
    """The precision forms' outer/inner structure, restated in numpy FP64: from
    an iterate Psi, the residual r = b(Psi) - A Psi (per cell, inflow from Psi's
    neighbours), then OCI sweeps on the correction (delta_j <- A_j^{-1} (r_j +
    inflow of delta from the neighbours, zero at the slab ends)), then Psi <-
    Psi + delta and a fresh residual.  A few refinements of a few inner sweeps
    reach the oracle's global direct solve of the step, as the plain OCI
    iteration does."""
    from oracle import brute
    p = W.random_slab(seed, J, N, G)
    o = Oracle(p, factor=False)
    A = [o.cell_matrix(j) for j in range(J)]
    ref = brute.solve_step(p, o.psi_prev)
    rng = np.random.default_rng(seed)
    Psi = rng.uniform(0.0, 1.0, size=(J, G, N, 4))
    n = 4 * N * G

    def inflow(D, j):
        """The inflow part of b_j taken from the array D (the A_j-independent rows)."""
        b = np.zeros((G, N, 4))
        for g in range(G):
            for m in range(N):
                mu = o.mu[m]
                if mu > 0 and j > 0:
                    b[g, m, 0] += mu * D[j - 1, g, m, 1]
                    b[g, m, 2] += mu * D[j - 1, g, m, 3]
                if mu < 0 and j < J - 1:
                    b[g, m, 1] += -mu * D[j + 1, g, m, 0]
                    b[g, m, 3] += -mu * D[j + 1, g, m, 2]
        return b.reshape(n)

    for _ in range(12):  # refinements
        r = np.stack([o.rhs(j, Psi) - A[j] @ Psi[j].reshape(n) for j in range(J)])
        delta = np.zeros_like(Psi)
        for _ in range(8):  # inner correction sweeps (block Jacobi)
            delta = np.stack([np.linalg.solve(A[j], r[j] + inflow(delta, j)).reshape(G, N, 4) for j in range(J)])
        Psi = Psi + delta
    assert np.abs(Psi - ref).max() < 1e-12 * np.abs(ref).max()
