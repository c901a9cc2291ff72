"""All FP64 sweeps of a step in one launch: the register form of the sweep
where every cell block fits on the GPU at once, as a cooperative grid (each
block writes its partial of ||Psi^{l+1} - Psi^l||^2, meets the others at a
bounded grid barrier and sums all partials) or, for at most 16 blocks, as one
thread-block cluster that keeps the iterate on chip and exchanges the block-edge
corners and the partials through distributed shared memory.  Both sum the same
partials in the same fixed order as the last block of a one-sweep launch, so the
iterates, the norms and the sweep counts of a step must equal those of one
launch per sweep bit for bit, and the oracle's sweep counts and flux within
1e-12 (Sec. 2.1, Algorithm 2).  Cases: one ragged block, many blocks with a
ragged last one, one and two groups, 2, 4 and 8 angles per thread, and the
two-group problem of the paper's GPU experiment (Sec. 3.2, Table 2)."""
import numpy as np
import pytest

from oracle import OCI, Oracle
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (seed, J, N, G, OCI_SWEEP_SHAPE "cells per block, angle chunks")
CASES = [(91, 40, 8, 1, "64,2"), (92, 1000, 16, 1, "64,4"), (93, 333, 8, 2, "32,2"),
         (94, 2049, 32, 1, "32,4"), (95, 500, 16, 1, "32,8"), (96, 6000, 16, 1, "16,4"),
         (98, 17, 16, 2, "16,4"), (99, 1024, 16, 2, "64,2"), (101, 300, 2, 3, "32,1"),
         (102, 200, 4, 2, "16,2"), (103, 700, 8, 2, "4,4")]
# OCI_SWEEP_MS: "grid" keeps the cooperative form, unset lets the cluster form take <= 16 blocks
FORMS = {"grid": "grid", "cluster": None}


def group_rel(a, b):
    return max(float(np.abs(a[:, g] - b[:, g]).max() / np.abs(b[:, g]).max()) for g in range(b.shape[1]))


def _steps(p, n, psi0=None):
    with oci.Solver(p) as s:
        info = s.info()
        if psi0 is not None:
            s.set_psi(psi0)
        sts = [s.step() for _ in range(n)]
        return info, sts, s.psi(), s.phi()


def _form(monkeypatch, form):
    if FORMS[form] is None:
        monkeypatch.delenv("OCI_SWEEP_MS", raising=False)
    else:
        monkeypatch.setenv("OCI_SWEEP_MS", FORMS[form])


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("seed,J,N,G,shape", CASES)
def test_one_launch_equals_one_launch_per_sweep(seed, J, N, G, shape, form, monkeypatch):
    monkeypatch.setenv("OCI_SWEEP_REG", "1")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", shape)
    cb = int(shape.split(",")[0])
    want = 2 if form == "cluster" and -(-J // cb) <= 16 else 1
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    _form(monkeypatch, form)
    ia, sa, psia, phia = _steps(p, 3)
    monkeypatch.setenv("OCI_SWEEP_MS", "0")
    ib, sb, psib, phib = _steps(p, 3)
    assert ia["sweep_kernel"] == ib["sweep_kernel"] == 1
    assert (ia["multi_sweep"], ib["multi_sweep"]) == (want, 0)
    for a, b in zip(sa, sb):
        assert a["status"] == b["status"] == 0
        assert (a["iters"], a["e"], a["rho"]) == (b["iters"], b["e"], b["rho"])
    assert np.array_equal(psia, psib) and np.array_equal(phia, phib)
    o = Oracle(p)
    for k in range(3):
        r = o.step(OCI)
        assert sa[k]["iters"] == r["iters"], (k, sa[k]["iters"], r["iters"])
    assert group_rel(phia, r["phi"]) < 1e-12


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("N,dt,delta2", [(16, 10.0, 0.05), (16, 10.0, 8.0), (32, 0.1, 0.25), (32, 10.0, 0.1)])
def test_table2_problem_in_one_launch_against_oracle(N, dt, delta2, form, monkeypatch):
    """Sec. 3.2, Table 2: J = 100 / delta2 cells, two groups with upscatter."""
    monkeypatch.setenv("OCI_SWEEP_REG", "1")
    _form(monkeypatch, form)
    p = W.rosa_two_group(delta2, N, dt).replace(tol=1e-10)
    r = Oracle(p, share_factors=True).step(OCI)
    with oci.Solver(p) as s:
        ms = s.info()["multi_sweep"]
        assert ms == 1 if form == "grid" else ms in (1, 2)
        st = s.step()
        assert st["status"] == 0 and st["iters"] == r["iters"], (st["iters"], r["iters"])
        assert group_rel(s.phi(), r["phi"]) < 1e-12


@pytest.mark.parametrize("form", list(FORMS))
def test_one_launch_starts_from_a_given_iterate(form, monkeypatch):
    """A step from an iterate set through oci_set_psi: the first sweep's norm
    uses it, as in one launch per sweep."""
    monkeypatch.setenv("OCI_SWEEP_REG", "1")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", "64,4")
    _form(monkeypatch, form)
    p = W.random_slab(97, 1000, 16, 1).replace(tol=1e-11)
    psi0 = W.random_guess(p, 5)
    ia, sa, psia, _ = _steps(p, 2, psi0)
    monkeypatch.setenv("OCI_SWEEP_MS", "0")
    ib, sb, psib, _ = _steps(p, 2, psi0)
    assert (ia["multi_sweep"], ib["multi_sweep"]) == (1 if form == "grid" else 2, 0)
    assert [(x["iters"], x["e"]) for x in sa] == [(x["iters"], x["e"]) for x in sb]
    assert np.array_equal(psia, psib)


def test_cluster_form_then_fixed_sweeps_on_the_same_handle(monkeypatch):
    """oci_iterate (one launch per sweep) after a step run by the cluster form
    continues from the iterate the cluster wrote back."""
    monkeypatch.setenv("OCI_SWEEP_REG", "1")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", "64,2")
    p = W.random_slab(100, 700, 8, 2).replace(tol=1e-11)
    with oci.Solver(p) as a:
        assert a.info()["multi_sweep"] == 2
        a.step()
        ea = a.iterate(3)
        psia = a.psi()
    monkeypatch.setenv("OCI_SWEEP_MS", "0")
    with oci.Solver(p) as b:
        b.step()
        eb = b.iterate(3)
        psib = b.psi()
    assert np.array_equal(ea, eb) and np.array_equal(psia, psib)


def test_too_many_blocks_keep_one_launch_per_sweep(monkeypatch):
    """2^18 cells in 16-cell blocks cannot all be resident: one launch per sweep."""
    monkeypatch.setenv("OCI_SWEEP_REG", "1")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", "16,4")
    p = W.slab_3region(c=0.9, tau=0.1, J=2 ** 18)
    with oci.Solver(p) as s:
        info = s.info()
        assert info["sweep_kernel"] == 1 and info["multi_sweep"] == 0
        assert s.step()["status"] == 0
