"""Fourier (von Neumann) analysis tools for the SCB x MB discretisation
(test infrastructure only).

Model problem: infinite homogeneous medium, one group, Sigma_t = 1, v = 1, so
that the cell optical thickness delta = Sigma dx gives dx = delta, the mean free
time tau = Sigma v dt gives dt = tau, and the scattering ratio c gives
Sigma_s = c.  tau = inf means steady state (no time-absorption terms).

An error mode f_{j} = a e^{i theta j} turns the lagged inflow of a cell into the
neighbour's corner value times e^{-+ i theta}:
  mu > 0: rows (kL, hL) receive mu * (kR, hR) of cell j-1  -> factor e^{-i theta}
  mu < 0: rows (kR, hR) receive |mu| * (kL, hL) of cell j+1 -> factor e^{+i theta}
With the within-cell operator L_c (Eq. Aj), the scattering matrix S (Eq.
scatter, reading: column-angle weight) and that inflow operator B(theta):
  T_OCI(theta) = (L_c - S)^{-1} B(theta)     (Sec. 2.3)
  T_SI(theta)  = (L_c - B(theta))^{-1} S     (Sec. 2.3)
and rho = max over theta of the largest |eigenvalue| (numpy.linalg.eigvals).
The time-march matrix of Sec. 2.2 (no scattering) maps psi_{k-1/2} (L, R) of a
mode to psi_{k+1/2} for one ordinate.
"""
from __future__ import annotations

import numpy as np


def _blocks(mu, delta, tau):
    alpha = 0.0 if np.isinf(tau) else delta / tau
    a = (abs(mu) + delta) / 2.0
    return np.array([[a, mu / 2, alpha / 2, 0.0],
                     [-mu / 2, a, 0.0, alpha / 2],
                     [-alpha, 0.0, alpha + a, mu / 2],
                     [0.0, -alpha, -mu / 2, alpha + a]])


def operators(N, delta, tau, c, theta):
    mu, w = np.polynomial.legendre.leggauss(N)
    n = 4 * N
    Lc = np.zeros((n, n), complex)
    S = np.zeros((n, n), complex)
    B = np.zeros((n, n), complex)
    for m in range(N):
        Lc[4 * m:4 * m + 4, 4 * m:4 * m + 4] = _blocks(mu[m], delta, tau)
        if mu[m] > 0:
            f = mu[m] * np.exp(-1j * theta)
            B[4 * m + 0, 4 * m + 1] = f
            B[4 * m + 2, 4 * m + 3] = f
        else:
            f = -mu[m] * np.exp(1j * theta)
            B[4 * m + 1, 4 * m + 0] = f
            B[4 * m + 3, 4 * m + 2] = f
        for nn in range(N):
            for p in range(4):
                S[4 * m + p, 4 * nn + p] = delta * c / 4.0 * w[nn]
    return Lc, S, B


def T_oci(N, delta, tau, c, theta):
    Lc, S, B = operators(N, delta, tau, c, theta)
    return np.linalg.solve(Lc - S, B)


def T_si(N, delta, tau, c, theta):
    Lc, S, B = operators(N, delta, tau, c, theta)
    return np.linalg.solve(Lc - B, S)


def spectral_radius(kind, N, delta, tau, c, n_theta=250, return_eig=False):
    thetas = np.linspace(0.0, 2 * np.pi, n_theta)
    f = T_oci if kind == "oci" else T_si
    best, lam = -1.0, None
    for th in thetas:
        ev = np.linalg.eigvals(f(N, delta, tau, c, th))
        k = int(np.argmax(np.abs(ev)))
        if abs(ev[k]) > best:
            best, lam = abs(ev[k]), ev[k]
    return (best, lam) if return_eig else best


def rho_si_flat(tau, c):
    """Closed form of the SI flat-mode (theta = 0) spectral radius: the MB pair
    (psi_k, psi_h) of an isotropic flat error obeys M (psi_k, psi_h) = c (old),
    M = [[1, 1/tau], [-2/tau, 1 + 2/tau]], whose eigenvalues are
    (1 + 1/tau) +- i/tau, so rho = c / sqrt((1 + 1/tau)^2 + 1/tau^2)."""
    if np.isinf(tau):
        return c
    return c / np.sqrt((1 + 1 / tau) ** 2 + 1 / tau ** 2)


def K_march(mu, delta, tau, theta):
    """2x2 amplification matrix psi_{k-1/2} -> psi_{k+1/2} of one ordinate for a
    mode e^{i theta j} in a non-scattering infinite medium (Sec. 2.2)."""
    alpha = delta / tau
    L = _blocks(mu, delta, tau).astype(complex)
    if mu > 0:
        L[0, 1] -= mu * np.exp(-1j * theta)
        L[2, 3] -= mu * np.exp(-1j * theta)
    else:
        L[1, 0] -= -mu * np.exp(1j * theta)
        L[3, 2] -= -mu * np.exp(1j * theta)
    K = np.zeros((2, 2), complex)
    for col in range(2):
        rhs = np.zeros(4, complex)
        rhs[col] = alpha / 2.0
        x = np.linalg.solve(L, rhs)
        K[:, col] = x[2:4]
    return K
