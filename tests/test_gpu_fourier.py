"""GPU batched Fourier tool (oci_fourier_rho) against the oracle's Fourier
analysis (numpy eigenvalues of the full 4N x 4N operators on the same theta
grid), and the SI flat-mode closed form."""
import numpy as np
import pytest

from oracle import fourier as F
from paper_2503_00264_gb300 import oci

pytestmark = pytest.mark.gpu

CASES = [(8, 0.1, 0.1, 0.9), (8, 1.0, 0.01, 0.99), (16, 0.01, 1.0, 0.5), (4, 10.0, 10.0, 1.0),
         (8, 0.5, np.inf, 0.9), (2, 0.3, 0.3, 0.0), (32, 0.1, 0.1, 0.9)]


@pytest.mark.parametrize("kind,name", [(oci.FOURIER_OCI, "oci"), (oci.FOURIER_SI, "si")])
def test_fourier_rho_matches_oracle(kind, name):
    for N in sorted({c[0] for c in CASES}):
        sub = [c for c in CASES if c[0] == N]
        got = oci.fourier_rho(kind, N, [c[1] for c in sub], [c[2] for c in sub], [c[3] for c in sub], n_theta=41)
        for (n_, d, t, c), g in zip(sub, got):
            ref = F.spectral_radius(name, N, d, t, c, n_theta=41)
            assert abs(g - ref) <= 1e-7 * max(ref, 1e-12) + 1e-14, (name, N, d, t, c, g, ref)


def test_fourier_si_flat_mode_closed_form():
    taus = np.array([0.01, 0.1, 1.0, 10.0])
    got = oci.fourier_rho(oci.FOURIER_SI, 8, np.full(4, 0.2), taus, np.full(4, 0.8), n_theta=1)
    ref = [F.rho_si_flat(t, 0.8) for t in taus]
    assert np.allclose(got, ref, rtol=1e-9)


def test_fourier_oci_trend_with_mean_free_time():
    """rho_OCI falls as the mean free time shrinks (the trend of Sec. 2.3 and Table 1)."""
    taus = np.array([10.0, 1.0, 0.1, 0.01])
    r = oci.fourier_rho(oci.FOURIER_OCI, 16, np.full(4, 0.1), taus, np.full(4, 0.99), n_theta=121)
    assert np.all(np.diff(r) < 0) and r[-1] < 0.1 * r[0]


def _rho_march_oracle(N, delta, tau, n_theta):
    mu, _ = np.polynomial.legendre.leggauss(N)
    best = 0.0
    for th in np.linspace(0.0, 2 * np.pi, n_theta):
        for m in mu:
            best = max(best, float(np.abs(np.linalg.eigvals(F.K_march(m, delta, tau, th))).max()))
    return best


@pytest.mark.parametrize("N", [2, 8, 16, 32])
def test_fourier_march_matches_oracle_time_march_matrix(N):
    """Sec. 2.2: the GPU's closed-form K (Eqs. eig1-4, K+ and K-) against the
    oracle's time-march matrix built from the discretisation by a 4x4 solve
    per ordinate, on the same theta grid."""
    deltas = np.array([0.01, 0.5, 2.0, 10.0, 0.1])
    taus = np.array([0.01, 0.3, 1.0, 100.0, 5.0])
    got = oci.fourier_rho(oci.FOURIER_MARCH, N, deltas, taus, None, n_theta=25)
    for d, t, g in zip(deltas, taus, got):
        ref = _rho_march_oracle(N, d, t, 25)
        assert abs(g - ref) <= 1e-12 * max(ref, 1e-300), (N, d, t, g, ref)


def test_fourier_march_flat_mode_and_stability():
    """theta = 0: the largest amplification is the MB one 1/(1 + tau + tau^2/2)
    (the same closed form pins the oracle's matrix); over a Fig.-3-shaped (tau, delta)
    grid at S16 with 75 wave numbers no |lambda_K| exceeds 1; steady state 0."""
    taus = np.array([0.01, 0.1, 1.0, 10.0])
    flat = oci.fourier_rho(oci.FOURIER_MARCH, 16, np.full(4, 0.3), taus, None, n_theta=1)
    assert np.allclose(flat, 1.0 / (1.0 + taus + taus ** 2 / 2), rtol=1e-12)
    tg, dg = np.meshgrid(np.logspace(-3, 3, 25), np.logspace(-3, 2, 21), indexing="ij")
    rho = oci.fourier_rho(oci.FOURIER_MARCH, 16, dg.ravel(), tg.ravel(), None, n_theta=75)
    assert np.all(rho <= 1.0 + 1e-12) and np.all(rho > 0.0)
    assert oci.fourier_rho(oci.FOURIER_MARCH, 8, [0.5], [np.inf], None, n_theta=9)[0] == 0.0
