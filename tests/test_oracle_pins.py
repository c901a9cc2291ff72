"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it relies on.  None of them re-types the oracle's
own formulas: the references are an independent global direct solve written
from Eqs. scb-mb-a..d (oracle/brute.py), library routines, closed forms,
invariants and exact finite-step properties.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import OCI, RB, SI, Oracle, balance_residual
from oracle import brute
from oracle import fourier as F
from paper_2503_00264_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
def test_gauss_legendre_matches_library(N):
    """Gauss-Legendre S_N set (Sec. 1 footnote) equals numpy's leggauss."""
    mu, w = oracle.gauss_legendre(N)
    x, ww = np.polynomial.legendre.leggauss(N)
    assert np.abs(mu - x).max() < 1e-14
    assert np.abs(w - ww).max() < 1e-14
    assert abs(w.sum() - 2.0) < 1e-14


# ---------------------------------------------- P1/P2: brute-force global solve
CASES = [
    (1, 1, 2, 1), (2, 5, 4, 1), (3, 12, 8, 1), (4, 7, 4, 2), (5, 9, 2, 3), (6, 16, 8, 2),
]


@pytest.mark.parametrize("seed,J,N,G", CASES)
def test_oci_converges_to_global_solve(seed, J, N, G):
    """Converged OCI (Eq. oci, Algorithm 2) equals the direct solve of the
    full SCB x MB system (Eqs. scb-mb-a..d + closures) over 3 steps, which pins
    L_c (Eq. Aj), b (Eq. rhs_sg), S (Eq. scatter, multigroup Eq. fullOCIlhs),
    the boundary inflow and the end-of-step carry."""
    p = W.random_slab(seed, J, N, G)
    o = Oracle(p)
    ref = brute.transient(p, 3)
    for k in range(3):
        r = o.step(OCI, tol=1e-12)
        assert r["status"] == 0
        assert _rel(r["Psi"], ref[k]) < 1e-11, k
        phi_ref = np.einsum("jgmp,m->jgp", ref[k], np.polynomial.legendre.leggauss(N)[1])
        assert _rel(r["phi"], phi_ref) < 1e-12


@pytest.mark.parametrize("seed,J,N,G", CASES)
def test_si_converges_to_global_solve(seed, J, N, G):
    """Converged SI (Algorithm 1, App. A, reading: Jacobi group coupling) has
    the same fixed point as the direct solve, hence as OCI."""
    p = W.random_slab(seed, J, N, G)
    o = Oracle(p, factor=False)
    ref = brute.transient(p, 2)
    for k in range(2):
        r = o.step(SI, tol=1e-12)
        assert r["status"] == 0
        assert _rel(r["Psi"], ref[k]) < 1e-11


def test_scatter_transfer_orientation_matters():
    """A transposed transfer matrix (sigma_s[g][gp] read as gp -> g) must be
    detected: with an asymmetric Sigma_s the two give different solutions."""
    p = W.random_slab(11, 6, 4, 3)
    ref = brute.solve_step(p, p.psi_init)
    q = p.replace(sigma_s=np.ascontiguousarray(np.swapaxes(p.sigma_s, 1, 2)))
    wrong = brute.solve_step(q, p.psi_init)
    assert _rel(wrong, ref) > 1e-3
    o = Oracle(p)
    r = o.step(OCI, tol=1e-12, guess=1)
    assert _rel(r["Psi"], ref) < 1e-11


# ---------------------------------------------------------- P3: particle balance
@pytest.mark.parametrize("seed,J,N,G", CASES[1:])
def test_balance_exact_on_direct_solution(seed, J, N, G):
    """Summing Eqs. scb-mb-a+b and scb-mb-c+d over corners, angles and cells
    telescopes the streaming terms to the boundary leakage: the exact discrete
    solution satisfies both balances per group to rounding."""
    p = W.random_slab(seed, J, N, G)
    o = Oracle(p, factor=False)
    psi_prev = o.psi_prev.copy()
    Psi = brute.solve_step(p, psi_prev)
    _, rel = balance_residual(o.balance(psi_prev, Psi))
    assert rel.max() < 1e-13


def test_balance_of_iterate_is_order_e():
    """An OCI iterate satisfies the balances to O(e_last)."""
    p = W.random_slab(21, 20, 8, 2)
    o = Oracle(p)
    r = o.step(OCI, tol=1e-6)
    res, rel = balance_residual(r["bal"])
    assert np.abs(res).max() < 50 * r["e"]
    r2 = Oracle(p).step(OCI, tol=1e-12)
    assert balance_residual(r2["bal"])[1].max() < 1e-10


def test_balance_detects_wrong_solution():
    p = W.random_slab(22, 10, 4, 1)
    o = Oracle(p, factor=False)
    Psi = brute.solve_step(p, o.psi_prev)
    Psi[3, 0, 1, 2] *= 1.01
    _, rel = balance_residual(o.balance(o.psi_prev, Psi))
    assert rel.max() > 1e-5


# ------------------------------------------------- P4: infinite-medium invariance
@pytest.mark.parametrize("G", [1, 3])
def test_uniform_infinite_medium_invariance(G):
    """Uniform material, isotropic psi_init = psi_inc = psi_inf with
    (diag Sigma_t - Sigma_s^T) psi_inf = Q/2: psi stays psi_inf every step
    (Eq. sn_nte with d/dt = d/dx = 0)."""
    rng = np.random.default_rng(5)
    J, N = 9, 8
    st = rng.uniform(1.0, 2.0, size=(1, G))
    ss = np.zeros((1, G, G))
    for gp in range(G):
        ss[0, gp] = rng.dirichlet(np.ones(G)) * 0.8 * st[0, gp]
    Qg = rng.uniform(0.5, 1.5, size=G)
    psi_inf = np.linalg.solve(np.diag(st[0]) - ss[0].T, Qg / 2)
    inc = np.repeat(psi_inf[:, None, None], N, axis=1).repeat(2, axis=2)
    p = W.Problem(J=J, N=N, G=G, n_mat=1, dx=rng.uniform(0.1, 0.5, J), mat=np.zeros(J, np.int32),
                  sigma_t=st, sigma_s=ss, v=rng.uniform(1, 3, G), dt=0.3,
                  Q=np.tile(Qg[None, :, None], (J, 1, 4)),
                  psi_init=np.tile(psi_inf[None, :, None, None], (J, 1, N, 2)),
                  inc_left=inc, inc_right=inc, tol=1e-14)
    o = Oracle(p)
    o.Psi[...] = psi_inf[None, :, None, None]
    for _ in range(3):
        r = o.step(OCI, tol=1e-12)
        assert r["status"] == 0
        assert np.abs(r["Psi"] - psi_inf[None, :, None, None]).max() < 1e-13
        assert r["e_hist"][0] < 1e-13      # the exact guess is a fixed point


# ------------------------------------------------------- P5: MB closed form
def test_mb_closed_form_uniform_transient():
    """Spatially uniform isotropic transient with the boundary set each step to
    the uniform solution: every step reduces to the multiple-balance pair
    (1/(v dt))(psi_h - psi_prev) + Sa psi_k = Q/2,
    (2/(v dt))(psi_h - psi_k) + Sa psi_h = Q/2   (Eqs. 2a, 2b), Sa = St - Ss."""
    J, N = 7, 4
    st, ssv, v, dt, Qv = 1.3, 0.6, 2.0, 0.25, 0.8
    sa = st - ssv
    M = np.array([[sa, 1 / (v * dt)], [-2 / (v * dt), 2 / (v * dt) + sa]])
    seq, prev = [], 0.3
    for k in range(5):
        pk, ph = np.linalg.solve(M, [Qv / 2 + prev / (v * dt), Qv / 2])
        seq.append((pk, ph))
        prev = ph
    p = W.Problem(J=J, N=N, G=1, n_mat=1, dx=np.full(J, 0.2), mat=np.zeros(J, np.int32),
                  sigma_t=[[st]], sigma_s=[[[ssv]]], v=[v], dt=dt, Q=np.full((J, 1, 4), Qv),
                  psi_init=np.full((J, 1, N, 2), 0.3), tol=1e-14)
    o = Oracle(p)
    for k in range(5):
        pk, ph = seq[k]
        inc = np.zeros((1, N, 2))
        inc[..., 0], inc[..., 1] = pk, ph
        o.set_boundary(inc, inc)
        r = o.step(OCI, tol=1e-14)
        assert np.abs(r["Psi"][..., 0:2] - pk).max() < 1e-12
        assert np.abs(r["Psi"][..., 2:4] - ph).max() < 1e-12


# --------------------------------------------------------- P6: c = 0 nilpotency
def test_c0_oci_exact_after_J_sweeps():
    """Without scattering a cell's solution depends only on its upstream
    neighbours; block Jacobi moves exact information one cell per sweep, so
    sweep J+1 reproduces sweep J bit for bit (e = 0) and the step stops there."""
    J, N = 20, 4
    p = W.Problem(J=J, N=N, G=1, n_mat=1, dx=np.full(J, 0.3), mat=np.zeros(J, np.int32),
                  sigma_t=[[1.0]], sigma_s=[[[0.0]]], v=[1.0], dt=0.5, Q=np.ones((J, 1, 4)),
                  inc_left=W.isotropic_inflow(1, N, 1.0, "left"), tol=0.0)
    r = Oracle(p).step(OCI, tol=0.0, guess=1)
    assert r["status"] == 0 and r["iters"] == J + 1 and r["e"] == 0.0
    assert np.all(r["e_hist"][:J] > 0)
    r2 = Oracle(p, factor=False).step(SI, tol=0.0, guess=1)
    assert r2["status"] == 0 and r2["iters"] == 2


# ---------------------------------------------------------- P7: per-cell residual
def test_cell_solve_residual():
    p = W.random_slab(31, 6, 8, 2)
    o = Oracle(p)
    Psi_l = W.random_guess(p, 1)
    out = o.cells(np.arange(p.J), Psi_l)
    for j in range(p.J):
        A = o.cell_matrix(j)
        b = o.rhs(j, Psi_l)
        assert np.linalg.norm(A @ out[j].ravel() - b) <= 1e-13 * np.linalg.norm(b)


# ------------------------------------------------ P8: linearity and mirror symmetry
def test_linearity_in_sources():
    p1 = W.random_slab(41, 8, 4, 2)
    p2 = W.random_slab(42, 8, 4, 2).replace(dx=p1.dx, mat=p1.mat, sigma_t=p1.sigma_t,
                                            sigma_s=p1.sigma_s, v=p1.v, dt=p1.dt)
    a, b = 0.7, -1.3
    p3 = p1.replace(Q=a * p1.Q + b * p2.Q, inc_left=a * p1.inc_left + b * p2.inc_left,
                    inc_right=a * p1.inc_right + b * p2.inc_right,
                    psi_init=a * p1.psi_init + b * p2.psi_init)
    r = [Oracle(q).step(OCI, tol=1e-12)["Psi"] for q in (p1, p2, p3)]
    assert _rel(r[2], a * r[0] + b * r[1]) < 1e-11


def test_mirror_symmetry():
    """Reversing the cells and mu -> -mu (swap L <-> R corners) maps the
    solution onto itself."""
    p = W.random_slab(51, 9, 8, 2)
    N = p.N
    rev = p.replace(dx=p.dx[::-1].copy(), mat=p.mat[::-1].copy(), Q=p.Q[::-1][..., [1, 0, 3, 2]].copy(),
                    psi_init=p.psi_init[::-1][:, :, ::-1][..., [1, 0]].copy(),
                    inc_left=p.inc_right[:, ::-1].copy(), inc_right=p.inc_left[:, ::-1].copy())
    a = Oracle(p).step(OCI, tol=1e-12)["Psi"]
    b = Oracle(rev).step(OCI, tol=1e-12)["Psi"]
    b_back = b[::-1][:, :, ::-1][..., [1, 0, 3, 2]]
    assert _rel(b_back, a) < 1e-11


# --------------------------------------------------------------- stop rule
def test_stop_rule_first_satisfying_iteration():
    """Sec. 2.1 / Algorithm 2: stop at the first l >= 1 with
    e_l < tol (1 - e_l / e_{l-1})."""
    p = W.random_slab(61, 30, 8, 1, c_max=0.99)
    tol = 1e-9
    r = Oracle(p).step(OCI, tol=tol)
    e = r["e_hist"]
    n = r["iters"]
    assert r["status"] == 0
    for l in range(1, n - 1):
        assert not (e[l] < tol * (1 - e[l] / e[l - 1]))
    assert e[n - 1] < tol * (1 - e[n - 1] / e[n - 2])
    assert abs(r["rho"] - e[n - 1] / e[n - 2]) < 1e-15


def test_noconv_does_not_commit():
    p = W.random_slab(62, 30, 8, 1, c_max=0.99)
    o = Oracle(p)
    prev = o.psi_prev.copy()
    r = o.step(OCI, tol=1e-14, max_iter=3)
    assert r["status"] == oracle.NOCONV and r["iters"] == 3
    assert np.array_equal(o.psi_prev, prev) and o.t == 0.0


# ------------------------------------------------ P9: Fourier analysis and trends
def _gold(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, *vals = line.split()
            rows[k] = [float(x) for x in vals]
    return rows


def test_si_fourier_matches_flat_mode_closed_form():
    for tau in (0.01, 0.1, 1.0, 10.0, np.inf):
        for c in (0.5, 0.99, 1.0):
            rho = F.spectral_radius("si", 8, 0.5, tau, c, n_theta=61)
            assert abs(rho - F.rho_si_flat(tau, c)) < 1e-12


def test_oci_fourier_table1_trends():
    """Table 1: steady state rho = 1 at c = 1 for every delta; in the transient
    rho falls as tau falls and as delta grows.  The printed table has the same
    ordering (its absolute values are not reproducible)."""
    g = _gold("table1_oci_rho.txt")
    taus = [np.inf, 10.0, 1.0, 0.1, 0.01]
    keys = ["SS", "10", "1", "0.1", "0.01"]
    ours = np.array([[F.spectral_radius("oci", 8, d, t, 1.0, n_theta=121) for d in (10.0, 1.0, 0.1)]
                     for t in taus])
    paper = np.array([g[k] for k in keys])
    assert np.abs(ours[0] - 1.0).max() < 1e-9
    for tab in (ours, paper):
        assert np.all(np.diff(tab[1:], axis=0) < 0)     # tau down -> rho down
        assert np.all(np.diff(tab[1:], axis=1) > 0)     # delta down -> rho up


def test_time_march_unconditionally_stable():
    """Sec. 2.2: sup |lambda_K| <= 1 over (tau, delta, theta, mu); the flat
    mode's eigenvalue is the MB amplification 1 / (1 + tau + tau^2/2)."""
    mu, _ = np.polynomial.legendre.leggauss(16)
    for tau in (0.01, 0.3, 1.0, 10.0, 1000.0):
        for delta in (0.01, 0.5, 10.0):
            for th in np.linspace(0, 2 * np.pi, 25):
                for m in mu:
                    assert np.abs(np.linalg.eigvals(F.K_march(m, delta, tau, th))).max() <= 1 + 1e-12
            lam = np.linalg.eigvals(F.K_march(mu[-1], delta, tau, 0.0))
            assert np.abs(lam - 1.0 / (1 + tau + tau ** 2 / 2)).min() < 1e-12


def test_table2_reading():
    """Table 2 reading: c_1 = (0.61789 + 0.92747)/1.5454 = 0.99997 as printed,
    and tau_2 = Sigma_2 v_2 dt = 2.2734 at dt = 10 (Fig. 6 caption)."""
    g = _gold("table2_rosa.txt")
    st, self_, other = g["sigma_t"], g["sigma_s_self"], g["sigma_s_other"]
    # out-scatter of group 1 = self + (1 -> 2)
    c1 = (self_[0] + other[1]) / st[0]
    assert abs(c1 - g["c_printed"][0]) < 1e-5
    assert abs(st[1] * g["v"][1] * 10.0 - g["tau2_dt10"][0]) < 1e-4
    assert abs(st[1] * g["v"][1] * 0.1 - g["tau2_dt0.1"][0]) < 1e-4
    p = W.rosa_two_group(1.0)
    assert p.sigma_s[0, 0, 1] == other[1] and p.sigma_s[0, 1, 0] == other[0]


@pytest.mark.slow
def test_measured_rate_matches_fourier_verification_problem():
    """Verification problem of Sec. 3.1 (delta = 0.25, tau = 1, c = 0.9, S8,
    random guess, no source): the empirical rate e_l / e_{l-1} averaged over the
    asymptotic iterations matches our Fourier rho (0.6403) within 2%."""
    g = _gold("verification_problem.txt")
    J = 1000
    p = W.Problem(J=J, N=8, G=1, n_mat=1, dx=np.full(J, g["dx"][0]), mat=np.zeros(J, np.int32),
                  sigma_t=[[g["sigma_t"][0]]], sigma_s=[[[g["c"][0] * g["sigma_t"][0]]]], v=[g["v"][0]],
                  dt=g["dt"][0], tol=g["tol"][0], max_iter=400)
    o = Oracle(p)
    o.Psi[...] = W.random_guess(p, 3)
    e = o.iterate(160)
    rate = np.exp(np.mean(np.log(e[100:160] / e[99:159])))
    rho = F.spectral_radius("oci", 8, 0.25, 1.0, 0.9)
    assert abs(rate - rho) / rho < 0.02


def test_iteration_counts_fall_with_mean_free_time():
    """Trend of Sec. 3.1: at fixed delta and c, OCI needs fewer
    iterations as tau shrinks, as the Fourier rho predicts."""
    J, N = 120, 8
    counts, rhos = [], []
    for tau in (10.0, 1.0, 0.1, 0.01):
        p = W.Problem(J=J, N=N, G=1, n_mat=1, dx=np.full(J, 0.3), mat=np.zeros(J, np.int32),
                      sigma_t=[[1.0]], sigma_s=[[[0.9]]], v=[1.0], dt=tau, Q=np.ones((J, 1, 4)), tol=1e-10)
        counts.append(Oracle(p).step(OCI)["iters"])
        rhos.append(F.spectral_radius("oci", N, 0.3, tau, 0.9, n_theta=61))
    assert all(a > b for a, b in zip(counts, counts[1:])), counts
    assert all(a > b for a, b in zip(rhos, rhos[1:])), rhos


# ------------------------------------------------- red-black ordering (block GS)
@pytest.mark.parametrize("seed,J,N,G", CASES[1:4])
def test_red_black_converges_to_global_solve(seed, J, N, G):
    """Red-black OCI has the fixed point of the discrete system (same as block
    Jacobi OCI); only the order of the cell solves differs."""
    p = W.random_slab(seed, J, N, G)
    o = Oracle(p)
    ref = brute.transient(p, 2)
    for k in range(2):
        r = o.step(RB, tol=1e-12)
        assert r["status"] == 0
        assert _rel(r["Psi"], ref[k]) < 1e-11


def test_red_black_rate_is_jacobi_rate_squared():
    """The cell coupling is block tridiagonal (block 2-cyclic), so red-black
    block Gauss-Seidel is consistently ordered and its asymptotic rate is the
    square of block Jacobi's (Young's theorem); measured on a long slab."""
    J = 400
    p = W.Problem(J=J, N=8, G=1, n_mat=1, dx=np.full(J, 0.1), mat=np.zeros(J, np.int32), sigma_t=[[1.0]],
                  sigma_s=[[[0.9]]], v=[1.0], dt=1.0, tol=1e-30, max_iter=400)
    rates = {}
    for method in (OCI, RB):
        o = Oracle(p)
        o.Psi[...] = W.random_guess(p, 4)
        e = o.iterate(160, method=method)
        rates[method] = np.exp(np.mean(np.log(e[120:160] / e[119:159])))
    assert abs(rates[RB] - rates[OCI] ** 2) < 0.02 * rates[OCI] ** 2, rates


def test_red_black_c0_exact_in_fewer_sweeps():
    """Without scattering information still moves one red-black pair of cells
    per half sweep in the direction of flight, so the exact solution is reached
    in at most about half the Jacobi sweep count."""
    J, N = 20, 4
    p = W.Problem(J=J, N=N, G=1, n_mat=1, dx=np.full(J, 0.3), mat=np.zeros(J, np.int32), sigma_t=[[1.0]],
                  sigma_s=[[[0.0]]], v=[1.0], dt=0.5, Q=np.ones((J, 1, 4)),
                  inc_left=W.isotropic_inflow(1, N, 1.0, "left"), tol=0.0)
    r = Oracle(p).step(RB, tol=0.0, guess=1)
    assert r["status"] == 0 and r["e"] == 0.0
    assert r["iters"] <= J // 2 + 2


# ------------------------------------- multigroup SI coupling (reading of App. A)
def _si_flat_iteration_matrix(st, ss, v, dt, coupling):
    """Iteration matrix of the spatially flat, isotropic SI error mode in an
    infinite medium, derived from the MB equations (Eqs. scb-mb-a..d summed over
    the two corners: streaming cancels for a flat mode).  Per group g the
    unknowns are the time-average and time-edge errors (e_k, e_h); with
    a_g = 1/(v_g dt) and the scattering source taken from the lagged iterate,
        Sigma_t,g e_k + a_g e_h            = sum_g' Sigma_s,g'->g e_k,g'(old)
        -2 a_g e_k + (Sigma_t,g + 2 a_g) e_h = sum_g' Sigma_s,g'->g e_h,g'(old)
    (an isotropic error has phi = 2 psi and the angular source is phi/2).
    coupling 'jacobi': every group's in-scatter from the lagged sweep (reading
    of App. A, all groups and angles in parallel); 'gauss_seidel': in-scatter
    from lower-index groups already updated in the same sweep."""
    G = len(st)
    M = np.zeros((2 * G, 2 * G))
    S = np.zeros((2 * G, 2 * G))
    for g in range(G):
        a = 1.0 / (v[g] * dt)
        M[2 * g:2 * g + 2, 2 * g:2 * g + 2] = [[st[g], a], [-2 * a, st[g] + 2 * a]]
        for gp in range(G):
            S[2 * g, 2 * gp] = S[2 * g + 1, 2 * gp + 1] = ss[gp][g]
    if coupling == "jacobi":
        return np.linalg.solve(M, S)
    low = np.zeros_like(S)
    for g in range(G):
        low[2 * g:2 * g + 2, :2 * g] = S[2 * g:2 * g + 2, :2 * g]
    return np.linalg.solve(M - low, S - low)


def test_si_flat_mode_matrix_reduces_to_one_group_closed_form():
    """For G = 1 the derived matrix has the closed-form radius of the pinned
    one-group flat mode, c / sqrt((1 + 1/tau)^2 + 1/tau^2)."""
    for tau in (0.05, 1.0, 7.0):
        for c in (0.3, 0.9):
            T = _si_flat_iteration_matrix([1.0], [[c]], [1.0], tau, "jacobi")
            assert abs(np.abs(np.linalg.eigvals(T)).max() - F.rho_si_flat(tau, c)) < 1e-14


@pytest.mark.parametrize("st,ss,v,dt", [
    ([1.0, 2.0], [[0.3, 0.6], [0.9, 0.5]], [1.0, 0.5], 1.0),
    ([1.0, 2.0], [[0.3, 0.6], [0.9, 0.5]], [1.0, 0.5], 10.0),
    ([1.0, 1.5, 2.5], [[0.2, 0.5, 0.2], [0.4, 0.3, 0.6], [0.3, 0.8, 1.0]], [3.0, 1.0, 0.3], 5.0),
])
def test_si_multigroup_rate_is_jacobi_over_groups(st, ss, v, dt):
    """Reading of the SI group update (App. A, Eq. app:si_update garbled):
    Jacobi over groups.  On a long uniform slab (300 mean free paths of the
    thinnest group) the oracle's measured asymptotic SI rate equals the radius
    of the derived flat-mode matrix with Jacobi coupling within 2%, while the
    Gauss-Seidel-over-groups radius of the same model misses it by more than 10%
    (strong up- and downscatter make the two readings far apart)."""
    G, J, N = len(st), 600, 8
    p = W.Problem(J=J, N=N, G=G, n_mat=1, dx=np.full(J, 0.5), mat=np.zeros(J, np.int32),
                  sigma_t=[st], sigma_s=[ss], v=v, dt=dt, tol=1e-30, max_iter=240)
    o = Oracle(p, factor=False)
    o.Psi[...] = W.random_guess(p, 7)
    e = o.iterate(240, method=SI)
    rate = (e[-1] / e[-121]) ** (1.0 / 120)
    rj = np.abs(np.linalg.eigvals(_si_flat_iteration_matrix(st, ss, v, dt, "jacobi"))).max()
    rg = np.abs(np.linalg.eigvals(_si_flat_iteration_matrix(st, ss, v, dt, "gauss_seidel"))).max()
    assert abs(rate - rj) < 0.02 * rj, (rate, rj)
    assert abs(rate - rg) > 0.10 * rg, (rate, rg)


def test_shared_factors_give_the_same_bits():
    """Factoring A_j once per distinct (material, dx) pair (the memory-saving
    mode used at full size) changes nothing: A_j depends on no other cell
    datum, so the iterates, norms and committed steps are bitwise equal to one
    factor per cell, for OCI and red-black OCI."""
    p = W.slab_3region(c=0.9, tau=0.3, J=3 * 40 + 7, N=8, region=40)
    for method in (OCI, RB):
        a, b = Oracle(p), Oracle(p, share_factors=True)
        assert b.n_slots == 3 and b.LU.shape[0] == 3
        for _ in range(2):
            ra, rb = a.step(method), b.step(method)
            assert ra["iters"] == rb["iters"]
            assert np.array_equal(ra["Psi"], rb["Psi"]) and np.array_equal(ra["e_hist"], rb["e_hist"])
    q = W.random_slab(8, 30, 4, 2)
    assert Oracle(q, share_factors=True).n_slots == 30
