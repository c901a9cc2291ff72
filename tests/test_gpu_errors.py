"""Failure paths of the C ABI, made on the host or by a bounded device wait
that is told to give up at once -- no GPU fault is involved.

  - OCI_E_TIMEOUT: the cooperative multi-sweep kernels (the FP32 inner sweeps
    and the FP64 register sweep where all its blocks fit) wait on a bounded
    grid barrier; with the test hook OCI_TEST_SPIN_LIMIT=0 every block that is
    not the last to arrive gives up without waiting, the kernel returns and the
    step ends with OCI_E_TIMEOUT, not committed.  The next step on the same
    handle, with the normal limit, matches the oracle.
  - OCI_E_NONFINITE: a NaN put into the iterate through oci_set_psi makes the
    convergence norm (Sec. 2.1) NaN; the step is not committed.
  - OCI_E_SINGULAR: no legal input gives a cell matrix a zero pivot in exact
    arithmetic (each A_j is nonsingular for a finite time step: the
    dx/(v dt) terms dominate its diagonal); finite widths and cross sections so
    large that the within-cell system overflows FP64 do, and setup reports it
    before any step."""
import numpy as np
import pytest

from oracle import OCI, Oracle
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("kernel,env", [("two", {"OCI_MX_INNER": "two", "OCI_SWEEP_SHAPE": "32,4"}),
                                        ("tiledp", {"OCI_MX_INNER": "tiledp", "OCI_SWEEP_SHAPE": "64,4"}),
                                        ("rb2", {"OCI_MX_RB": "2", "OCI_SWEEP_SHAPE": "64,4"}),
                                        ("rb", {"OCI_MX_RB": "1", "OCI_SWEEP_SHAPE": "64,4"}),
                                        ("fp64", {"OCI_SWEEP_REG": "1", "OCI_SWEEP_SHAPE": "64,4"})])
def test_grid_barrier_timeout_returns_status_and_handle_recovers(kernel, env, monkeypatch):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    p = W.random_slab(81, 4000, 16, 1).replace(tol=1e-11)
    psi0 = W.random_guess(p, 3)
    with oci.Solver(p, precision=oci.FP64 if kernel == "fp64" else oci.FP32_IR) as s:
        if kernel.startswith("rb"):
            s.set_ordering(oci.ORDER_RED_BLACK)
        if kernel == "fp64":  # all FP64 sweeps of the step in one cooperative launch
            assert s.info()["multi_sweep"] == 1
        pp0, t0 = s.state()
        s.set_psi(psi0)
        monkeypatch.setenv("OCI_TEST_SPIN_LIMIT", "0")
        with pytest.raises(oci.OCIError) as ei:
            s.step()
        assert ei.value.code == oci.E_TIMEOUT
        pp1, t1 = s.state()
        assert t1 == t0 and np.array_equal(pp0, pp1)  # not committed
        monkeypatch.delenv("OCI_TEST_SPIN_LIMIT")
        s.set_psi(psi0)
        st = s.step()
        o = Oracle(p)
        o.Psi[...] = psi0
        from oracle import RB
        r = o.step(RB if kernel.startswith("rb") else OCI)
        assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2, (st["iters"], r["iters"])
        assert rel(s.phi(), r["phi"]) < 1e-10


def test_spin_limit_hook_is_ignored_without_the_switch(monkeypatch):
    """Without OCI_TEST_HOOKS=1 the spin-limit override has no effect."""
    monkeypatch.setenv("OCI_MX_INNER", "two")
    p = W.random_slab(82, 3000, 16, 1).replace(tol=1e-11)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        monkeypatch.delenv("OCI_TEST_HOOKS")
        monkeypatch.setenv("OCI_TEST_SPIN_LIMIT", "0")
        st = s.step()
        assert st["status"] == 0


@pytest.mark.parametrize("precision", [oci.FP64, oci.FP32_IR])
def test_nan_iterate_gives_nonfinite_and_is_not_committed(precision):
    p = W.random_slab(83, 300, 8, 2).replace(tol=1e-11)
    psi = W.random_guess(p, 4)
    with oci.Solver(p, precision=precision) as s:
        pp0, t0 = s.state()
        bad = psi.copy()
        bad[123, 1, 5, 2] = np.nan
        s.set_psi(bad)
        with pytest.raises(oci.OCIError) as ei:
            s.step()
        assert ei.value.code == oci.E_NONFINITE
        assert b"not finite" in s.L.oci_last_error()
        pp1, t1 = s.state()
        assert t1 == t0 and np.array_equal(pp0, pp1)
        s.set_psi(psi)
        st = s.step()
        o = Oracle(p)
        o.Psi[...] = psi
        r = o.step(OCI)
        assert st["status"] == 0
        assert rel(s.phi(), r["phi"]) < (1e-12 if precision == oci.FP64 else 1e-10)


@pytest.mark.parametrize("solver", [oci.SOLVER_STRUCTURED, oci.SOLVER_DENSE_LU])
def test_overflowing_cell_system_is_reported_singular(solver):
    # dx/4 * Sigma_s = 2.5e309 overflows: the within-cell scalar-flux system
    # has infinite entries in its first pivot column (checked on the CPU)
    p = W.random_slab(84, 20, 4, 1).replace(dx=np.full(20, 1e10), sigma_s=np.full((2, 1, 1), 1e300))
    with pytest.raises(oci.OCIError) as ei:
        oci.Solver(p, solver=solver)
    assert ei.value.code == oci.E_SINGULAR
