"""Multi-step transients through oci_solve_transient (one ABI call, the phi of
every step written out) for each form against the oracle's step-by-step
transient: plain FP64, FP32_IR, red-black FP64 and FP32_IR, GMRES; plus the
mixed red-black form's uncommitted NOCONV and a batch of minimum-order slabs."""
import numpy as np
import pytest

from oracle import OCI, RB, Oracle
from oracle import brute
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


FORMS = [("fp64", oci.FP64, None, 1e-12, 0), ("fp32ir", oci.FP32_IR, None, 1e-10, 2),
         ("rb_fp64", oci.FP64, "rb", 1e-12, 0), ("rb_fp32ir", oci.FP32_IR, "rb", 1e-10, 2)]


@pytest.mark.parametrize("name,prec,order,tol_phi,slack", FORMS)
def test_solve_transient_matches_oracle(name, prec, order, tol_phi, slack):
    p = W.random_slab(121, 150, 8, 2).replace(tol=1e-11)
    o = Oracle(p)
    n = 4
    with oci.Solver(p, precision=prec) as s:
        if order == "rb":
            s.set_ordering(oci.ORDER_RED_BLACK)
        phi = np.zeros((n, p.J, p.G, 4))
        sts = s.solve_transient(n, phi)
        for k in range(n):
            r = o.step(RB if order == "rb" else OCI)
            assert sts[k]["status"] == 0
            assert abs(sts[k]["iters"] - r["iters"]) <= slack, (k, sts[k]["iters"], r["iters"])
            assert rel(phi[k], r["phi"]) < tol_phi, k
            assert abs(sts[k]["t"] - o.t) < 1e-12
            assert max(sts[k]["balance_rel"]) < 1e-9


def test_gmres_transient_matches_direct_solves():
    p = W.random_slab(122, 14, 4, 2).replace(tol=1e-13, max_iter=5000)
    ref = brute.transient(p, 4)
    with oci.Solver(p) as s:
        s.set_acceleration(oci.ACCEL_GMRES, restart=8, residual_factor=0.01)
        phi = np.zeros((4, p.J, p.G, 4))
        sts = s.solve_transient(4, phi)
        for k in range(4):
            mu, w = np.polynomial.legendre.leggauss(p.N)
            phi_ref = np.einsum("jgmp,m->jgp", ref[k], w)
            assert sts[k]["status"] == 0
            assert rel(phi[k], phi_ref) < 1e-10, k
            assert max(sts[k]["balance_rel"]) < 1e-9


def test_fp32_red_black_noconv_not_committed():
    p = W.random_slab(123, 80, 8, 1, c_max=0.99).replace(tol=1e-14, max_iter=3)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        s.set_ordering(oci.ORDER_RED_BLACK)
        pp0, t0 = s.state()
        with pytest.raises(oci.OCIError) as ei:
            s.step()
        assert ei.value.code == oci.E_NOCONV
        pp1, t1 = s.state()
        assert t1 == t0 and np.array_equal(pp0, pp1)


@pytest.mark.parametrize("prec", [oci.FP64, oci.FP32_IR])
def test_batch_minimum_order_slabs(prec):
    """S2 slabs (one ordinate each way) of 1 to 300 cells in one batch."""
    probs = [W.random_slab(130 + i, J, 2, G).replace(tol=1e-11)
             for i, (J, G) in enumerate([(1, 1), (2, 2), (37, 1), (300, 3), (129, 1)])]
    orcs = [Oracle(q) for q in probs]
    with oci.BatchSolver(probs, precision=prec) as b:
        for k in range(2):
            sts = b.step()
            for i, (q, o) in enumerate(zip(probs, orcs)):
                r = o.step(OCI)
                assert sts[i]["status"] == 0
                slack = 0 if prec == oci.FP64 else (3 if q.J == 1 else 2)
                assert abs(sts[i]["iters"] - r["iters"]) <= slack, (i, k)
                assert rel(b.phi(i), r["phi"]) < (1e-12 if prec == oci.FP64 else 1e-10)
