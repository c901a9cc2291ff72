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
