"""Seeded synthetic slab problems shaped like the paper's workloads.

This module only generates inputs (cross sections, widths, sources, boundary
values, initial iterates).  It holds none of the method's arithmetic and imports
nothing else from this package, so the CUDA path and the CPU oracle can both use
it without sharing code.

Field meanings follow the problem statement of the paper (Sec. 2.1, Eq. sn_nte,
Table 2):

    J, N, G, n_mat        cells, S_N order (even), groups, materials
    dx[J]                 cell widths (> 0)
    mat[J]                material index of each cell
    sigma_t[n_mat][G]     total cross section Sigma_t,g
    sigma_s[n_mat][G][G]  sigma_s[m][gp][g] = Sigma_s,gp->g (P0 transfer)
    v[G]                  particle speed per group
    Q[J][G][4]            isotropic total emission per corner and time level
                          (kL, kR, hL, hR); the angular source is Q/2
    dt                    time step
    psi_init[J][G][N][2]  initial angular flux at corners (L, R)
    inc_left[G][N][2]     incident angular flux for mu > 0 at x = 0
                          (time average over the step, value at the step end)
    inc_right[G][N][2]    incident angular flux for mu < 0 at x = X
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 20250301

GUESS_PREV = 0
GUESS_ZERO = 1


@dataclasses.dataclass
class Problem:
    J: int
    N: int
    G: int
    n_mat: int
    dx: np.ndarray
    mat: np.ndarray
    sigma_t: np.ndarray
    sigma_s: np.ndarray
    v: np.ndarray
    dt: float
    Q: Optional[np.ndarray] = None
    psi_init: Optional[np.ndarray] = None
    inc_left: Optional[np.ndarray] = None
    inc_right: Optional[np.ndarray] = None
    tol: float = 1e-10
    max_iter: int = 10000
    guess: int = GUESS_PREV
    name: str = ""

    def __post_init__(self):
        self.dx = np.ascontiguousarray(self.dx, dtype=np.float64).reshape(self.J)
        self.mat = np.ascontiguousarray(self.mat, dtype=np.int32).reshape(self.J)
        self.sigma_t = np.ascontiguousarray(self.sigma_t, dtype=np.float64).reshape(self.n_mat, self.G)
        self.sigma_s = np.ascontiguousarray(self.sigma_s, dtype=np.float64).reshape(self.n_mat, self.G, self.G)
        self.v = np.ascontiguousarray(self.v, dtype=np.float64).reshape(self.G)
        if self.Q is not None:
            self.Q = np.ascontiguousarray(self.Q, dtype=np.float64).reshape(self.J, self.G, 4)
        if self.psi_init is not None:
            self.psi_init = np.ascontiguousarray(self.psi_init, dtype=np.float64).reshape(self.J, self.G, self.N, 2)
        if self.inc_left is not None:
            self.inc_left = np.ascontiguousarray(self.inc_left, dtype=np.float64).reshape(self.G, self.N, 2)
        if self.inc_right is not None:
            self.inc_right = np.ascontiguousarray(self.inc_right, dtype=np.float64).reshape(self.G, self.N, 2)

    @property
    def unknowns(self) -> int:
        return 4 * self.N * self.G * self.J

    def replace(self, **kw) -> "Problem":
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        d.update(kw)
        return Problem(**d)


def _rng(config_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id + 1000 * salt))


def gauss_legendre_mu_sign(N: int) -> np.ndarray:
    """Sign pattern of the ascending Gauss-Legendre ordinates: first N/2 are
    negative, the last N/2 positive (N even).  Used only to shape boundary
    inputs; no quadrature arithmetic here."""
    s = np.ones(N)
    s[: N // 2] = -1.0
    return s


def isotropic_inflow(G: int, N: int, value: float, side: str) -> np.ndarray:
    """Incident angular flux `value` on every inward direction of one side."""
    inc = np.zeros((G, N, 2))
    sgn = gauss_legendre_mu_sign(N)
    inward = sgn > 0 if side == "left" else sgn < 0
    inc[:, inward, :] = value
    return inc


# ----------------------------------------------------------------------------
# Workloads.
# ----------------------------------------------------------------------------
def slab_64_cells(steps_note: bool = True) -> Problem:
    """64 uniform cells, dx = 0.1, S8, Sigma_t = 1, Sigma_s = 0.5, v = 1,
    dt = 0.1, zero initial flux, isotropic incident angular flux 1 on the left,
    vacuum on the right, tol 1e-8 (run for 10 steps)."""
    J, N, G = 64, 8, 1
    return Problem(
        J=J, N=N, G=G, n_mat=1,
        dx=np.full(J, 0.1), mat=np.zeros(J, np.int32),
        sigma_t=np.array([[1.0]]), sigma_s=np.array([[[0.5]]]), v=np.array([1.0]),
        dt=0.1, Q=None, psi_init=None,
        inc_left=isotropic_inflow(G, N, 1.0, "left"), inc_right=None,
        tol=1e-8, max_iter=10000, name="slab64_S8_G1",
    )


SLAB3_DELTAS = (0.01, 0.1, 1.0)
SLAB3_C = (0.5, 0.9, 0.99)
SLAB3_TAU = (0.01, 0.1, 1.0, 10.0)


def slab_3region(c: float = 0.9, tau: float = 1.0, J: int = 2 ** 18, N: int = 16,
                 region: int = 1024, ragged: bool = False, seed_salt: int = 0) -> Problem:
    """One group, S16, J cells in 3 repeating material regions of `region` cells
    (cell j in material (j // region) % 3) with optical thickness per cell
    delta in {0.01, 0.1, 1} (Sigma_t = 1 so dx = delta), scattering ratio c shared
    by all regions, v = 1 and dt = tau (mean free time Sigma_t v dt = tau),
    uniform unit source, zero initial flux, vacuum on both sides.
    `ragged=True` jitters every cell width by U(0.9, 1.1) so that no two cells
    share a local matrix."""
    G = 1
    mat = ((np.arange(J) // region) % 3).astype(np.int32)
    dx = np.array(SLAB3_DELTAS)[mat].copy()
    if ragged:
        dx = dx * _rng(2, seed_salt).uniform(0.9, 1.1, size=J)
    sig_t = np.ones((3, 1))
    sig_s = np.full((3, 1, 1), c)
    return Problem(
        J=J, N=N, G=G, n_mat=3, dx=dx, mat=mat, sigma_t=sig_t, sigma_s=sig_s,
        v=np.array([1.0]), dt=float(tau), Q=np.ones((J, G, 4)),
        psi_init=None, inc_left=None, inc_right=None, tol=1e-10, max_iter=20000,
        name=f"slab3_S{N}_G1_J{J}_c{c}_tau{tau}" + ("_ragged" if ragged else ""),
    )


def multigroup_scatter(rng: np.random.Generator, sigma_t: np.ndarray, c_lo: float = 0.5,
                       c_hi: float = 0.95) -> np.ndarray:
    """P0 transfer matrix sigma_s[gp][g] for one material: the row sum of source
    group gp is c_gp * Sigma_t,gp with c ~ U[c_lo, c_hi]; 5% of it goes to
    upscatter g < gp split proportional to 2^-(gp-g); 95% to g >= gp with a self
    share U[0.3, 0.6] and the rest proportional to 2^-(g-gp).  Rows without an
    up (gp = 0) or down (gp = G-1) target fold that share into self-scatter."""
    G = sigma_t.shape[0]
    S = np.zeros((G, G))
    for gp in range(G):
        total = rng.uniform(c_lo, c_hi) * sigma_t[gp]
        up_share = 0.05 if gp > 0 else 0.0
        self_frac = rng.uniform(0.3, 0.6)
        down_targets = list(range(gp + 1, G))
        down_share = 0.95 * (1 - self_frac) if down_targets else 0.0
        self_share = 1.0 - up_share - down_share
        S[gp, gp] = self_share * total
        if gp > 0:
            wts = np.array([2.0 ** -(gp - g) for g in range(gp)])
            S[gp, :gp] = up_share * total * wts / wts.sum()
        if down_targets:
            wts = np.array([2.0 ** -(g - gp) for g in down_targets])
            S[gp, gp + 1:] = down_share * total * wts / wts.sum()
    return S


def slab_multigroup(J: int = 2 ** 16, N: int = 16, G: int = 8, n_mat: int = 4, region: int = 1024,
                    dx: float = 0.1, dt: float = 1e-6, seed_salt: int = 0) -> Problem:
    """G groups, S16, J cells, n_mat materials in cycling blocks of `region`
    cells; Sigma_t,g ~ U[0.5, 5]; P0 scattering per `multigroup_scatter`
    (row sums c in [0.5, 0.95], mostly downscatter, 5% upscatter); v_g
    log-spaced from 1e7 (group 0) down to 1e2; no fission; unit source, zero
    initial flux, vacuum."""
    rng = _rng(3, seed_salt)
    sig_t = rng.uniform(0.5, 5.0, size=(n_mat, G))
    sig_s = np.stack([multigroup_scatter(rng, sig_t[m]) for m in range(n_mat)])
    v = np.logspace(7, 2, G)
    mat = ((np.arange(J) // region) % n_mat).astype(np.int32)
    return Problem(
        J=J, N=N, G=G, n_mat=n_mat, dx=np.full(J, dx), mat=mat, sigma_t=sig_t, sigma_s=sig_s,
        v=v, dt=dt, Q=np.ones((J, G, 4)), psi_init=None, inc_left=None, inc_right=None,
        tol=1e-10, max_iter=20000, name=f"multigroup_S{N}_G{G}_J{J}",
    )


def rosa_two_group(delta2: float = 1.0, N: int = 16, dt: float = 0.1, L: float = 100.0) -> Problem:
    """Two-group problem of the paper's Table 2 (L = 100, vacuum, psi0 = 0,
    Q = 1): Sigma = (1.5454, 0.45468), self scatter (0.61789, 0.0072534),
    in-scatter from the other group Sigma_s,2->1 = 0.38211 and
    Sigma_s,1->2 = 0.92747, v = (1, 0.5).  delta2 = Sigma_2 dx sets the width."""
    sig_t = np.array([[1.5454, 0.45468]])
    S = np.array([[[0.61789, 0.92747],    # from group 1: to 1, to 2
                   [0.38211, 0.0072534]]])  # from group 2: to 1, to 2
    dxv = delta2 / 0.45468
    J = max(1, int(round(L / dxv)))
    return Problem(
        J=J, N=N, G=2, n_mat=1, dx=np.full(J, L / J), mat=np.zeros(J, np.int32),
        sigma_t=sig_t, sigma_s=S, v=np.array([1.0, 0.5]), dt=dt, Q=np.ones((J, 2, 4)),
        tol=1e-10, max_iter=200000, name=f"rosa_S{N}_dt{dt}_delta{delta2}",
    )


def random_slab(seed: int, J: int, N: int, G: int, n_mat: int = 2, *, c_max: float = 0.95,
                source: bool = True, inflow: bool = True, init: bool = True,
                dt: Optional[float] = None) -> Problem:
    """Small random slab for parity and pin tests: random widths, materials,
    cross sections (Sigma_s row sums below c_max * Sigma_t), speeds, sources,
    inflows and initial fluxes."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 7919 * seed + 17))
    sig_t = rng.uniform(0.5, 3.0, size=(n_mat, G))
    S = np.zeros((n_mat, G, G))
    for m in range(n_mat):
        raw = rng.uniform(0.0, 1.0, size=(G, G))
        for gp in range(G):
            S[m, gp] = raw[gp] / raw[gp].sum() * rng.uniform(0.1, c_max) * sig_t[m, gp]
    return Problem(
        J=J, N=N, G=G, n_mat=n_mat,
        dx=rng.uniform(0.05, 0.6, size=J), mat=rng.integers(0, n_mat, size=J).astype(np.int32),
        sigma_t=sig_t, sigma_s=S, v=rng.uniform(0.5, 4.0, size=G),
        dt=float(rng.uniform(0.05, 2.0)) if dt is None else dt,
        Q=rng.uniform(0.0, 2.0, size=(J, G, 4)) if source else None,
        psi_init=rng.uniform(0.0, 1.0, size=(J, G, N, 2)) if init else None,
        inc_left=rng.uniform(0.0, 1.5, size=(G, N, 2)) if inflow else None,
        inc_right=rng.uniform(0.0, 1.5, size=(G, N, 2)) if inflow else None,
        tol=1e-13, max_iter=20000, name=f"random_{seed}_J{J}_N{N}_G{G}",
    )


def batch_of_slabs(n: int = 256, seed_salt: int = 0, j_lo: int = 1024, j_hi: int = 65536,
                   Ns=(4, 8, 16, 32), Gs=(1, 4)) -> list:
    """Independent slabs of uneven size: J_s ~ U_int[j_lo, j_hi], N_s from Ns,
    G_s from Gs; 1-4 materials each with Sigma_t ~ U[0.5, 5], c ~ U[0.3, 0.99]
    and a width per material dx ~ U[0.01, 1]/Sigma_t (shared within the
    material); speeds v = 1 (G = 1) or log-spaced 1e7..1e2 (G = 4); the largest
    mean free time max Sigma_t v dt over groups and materials is
    tau ~ logU[0.01, 10]; unit source, vacuum; tol 1e-10."""
    rng = _rng(5, seed_salt)
    out = []
    for s in range(n):
        J = int(rng.integers(j_lo, j_hi + 1))
        N = int(rng.choice(Ns))
        G = int(rng.choice(Gs))
        nm = int(rng.integers(1, 5))
        sig_t = rng.uniform(0.5, 5.0, size=(nm, G))
        S = np.zeros((nm, G, G))
        for m in range(nm):
            if G == 1:
                S[m, 0, 0] = rng.uniform(0.3, 0.99) * sig_t[m, 0]
            else:
                S[m] = multigroup_scatter(rng, sig_t[m], 0.3, 0.99)
        widths = rng.uniform(0.01, 1.0, size=nm) / sig_t[:, 0]
        mat = rng.integers(0, nm, size=J).astype(np.int32)
        tau = float(np.exp(rng.uniform(np.log(0.01), np.log(10.0))))
        v = np.ones(G) if G == 1 else np.logspace(7, 2, G)
        dt = tau / float((sig_t * v[None, :]).max())
        out.append(Problem(
            J=J, N=N, G=G, n_mat=nm, dx=widths[mat], mat=mat, sigma_t=sig_t, sigma_s=S,
            v=v, dt=dt, Q=np.ones((J, G, 4)), tol=1e-10, max_iter=20000,
            name=f"batch{s}_J{J}_N{N}_G{G}"))
    return out


def random_guess(p: Problem, seed: int = 0) -> np.ndarray:
    """Uniform [0, 1] initial iterate Psi[J][G][N][4] (the paper's verification
    problem starts from such a guess)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4242 + seed))
    return rng.uniform(0.0, 1.0, size=(p.J, p.G, p.N, 4))
