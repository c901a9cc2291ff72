"""Krylov (GMRES) acceleration of the FP64 OCI step: the same fixed point as
plain OCI (the exact discrete step from a global direct solve, and the oracle's
converged OCI step), fewer sweeps where OCI converges slowly, uncommitted
NOCONV, argument checks."""
import numpy as np
import pytest

from oracle import OCI, Oracle
from oracle import brute
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("seed,J,N,G,restart", [(111, 12, 4, 1, 20), (112, 9, 4, 2, 5), (113, 20, 8, 1, 1)])
def test_gmres_step_equals_direct_solve(seed, J, N, G, restart):
    """Tiny slabs: three GMRES steps against the exact discrete steps (global
    dense solve of the balance equations), within 1e-10."""
    p = W.random_slab(seed, J, N, G).replace(tol=1e-13, max_iter=5000)
    ref = brute.transient(p, 3)
    with oci.Solver(p) as s:
        s.set_acceleration(oci.ACCEL_GMRES, restart=restart, residual_factor=0.01)
        for k in range(3):
            st = s.step()
            assert st["status"] == 0 and st["rho"] == 0.0
            assert rel(s.psi(), ref[k]) < 1e-10, k


def test_gmres_matches_oracle_converged_step():
    """Three regions of 1024 cells (delta 0.01 / 0.1 / 1), c = 0.99, tau = 1:
    plain OCI contracts at ~0.98 per sweep (thin region).  GMRES(20) reaches the
    oracle's converged step; it takes no more sweeps than plain OCI (only a few
    percent fewer: OCI's slow modes in thin cells are streaming modes spread
    over the complex plane, not a cluster a Krylov polynomial can remove)."""
    p = W.slab_3region(c=0.99, tau=1.0, J=3072).replace(max_iter=20000)
    o = Oracle(p)
    r = o.step(OCI)
    with oci.Solver(p) as s:
        s.set_acceleration(oci.ACCEL_GMRES, restart=20, residual_factor=0.01)
        st = s.step()
        assert st["status"] == 0
        assert st["iters"] <= 1.05 * r["iters"], (st["iters"], r["iters"])
        assert rel(s.phi(), r["phi"]) < 1e-9
        assert max(st["balance_rel"]) < 1e-9
        s.set_acceleration(oci.ACCEL_NONE)
        st2 = s.step()  # plain OCI again on the next step
        assert st2["status"] == 0


def test_gmres_noconv_not_committed():
    p = W.random_slab(115, 60, 8, 1, c_max=0.99, dt=50.0).replace(tol=1e-14, max_iter=4)
    with oci.Solver(p) as s:
        s.set_acceleration(oci.ACCEL_GMRES, restart=3)
        pp0, t0 = s.state()
        with pytest.raises(oci.OCIError) as ei:
            s.step()
        assert ei.value.code == oci.E_NOCONV
        pp1, t1 = s.state()
        assert t1 == t0 and np.array_equal(pp0, pp1)


def test_gmres_argument_checks():
    p = W.random_slab(116, 20, 4, 1)
    with oci.Solver(p) as s:
        for args in ((7, 20, 0.05), (oci.ACCEL_GMRES, 0, 0.05), (oci.ACCEL_GMRES, 33, 0.05),
                     (oci.ACCEL_GMRES, 20, 0.0), (oci.ACCEL_GMRES, 20, 1.5)):
            assert s.L.oci_set_acceleration(s.h, *args) == oci.E_INVAL
        s.set_ordering(oci.ORDER_RED_BLACK)
        assert s.L.oci_set_acceleration(s.h, oci.ACCEL_GMRES, 20, 0.05) == oci.E_INVAL
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        assert s.L.oci_set_acceleration(s.h, oci.ACCEL_GMRES, 20, 0.05) == oci.E_INVAL
