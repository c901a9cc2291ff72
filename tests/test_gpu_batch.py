"""Batched form (many slabs, one graph launch per time step) against the FP64
oracle slab by slab: identical sweep counts, scalar flux within 1e-12; the
mixed-precision batched form within 1e-10 and a sweep count within the
refinement slack of the single-slab mixed form."""
import numpy as np
import pytest

from oracle import OCI, Oracle
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_batch_matches_oracle_per_slab():
    specs = [(41, 50, 4, 1), (42, 130, 8, 1), (43, 257, 8, 2), (44, 1, 4, 1), (45, 400, 16, 1), (46, 33, 8, 2),
             (47, 128, 4, 3), (48, 77, 8, 1)]
    probs = [W.random_slab(*sp).replace(tol=1e-11) for sp in specs]
    orcs = [Oracle(p) for p in probs]
    with oci.BatchSolver(probs) as b:
        for k in range(3):
            sts = b.step()
            for i, (p, o) in enumerate(zip(probs, orcs)):
                r = o.step(OCI)
                assert sts[i]["status"] == 0
                assert sts[i]["iters"] == r["iters"], (i, k, sts[i]["iters"], r["iters"])
                assert rel(b.phi(i), r["phi"]) < 1e-12
                assert rel(b.psi(i), r["Psi"]) < 1e-11
                assert np.abs(b.balance(i) - r["bal"]).max() <= 1e-11 * np.abs(r["bal"]).max()


def test_batch_uneven_slabs_match_single_slab_path():
    """64 slabs shaped like the 256-slab batch (N in {4,8,16,32}, G in {1,4},
    1-4 materials, random widths and mean free times), J in [1k, 4k]."""
    probs = [p.replace(max_iter=3000) for p in W.batch_of_slabs(64, j_lo=1024, j_hi=4096)]
    with oci.BatchSolver(probs) as b:
        sts = b.step(allow_noconv=True)
        for i in (0, 7, 21, 40, 63):
            with oci.Solver(probs[i]) as s:
                st = s.step(allow_noconv=True)
                assert st["status"] == sts[i]["status"]
                assert st["iters"] == sts[i]["iters"]
                if st["status"] == 0:
                    assert rel(b.phi(i), s.phi()) < 1e-12
        ok = [st for st in sts if st["status"] == 0]
        assert len(ok) > 32
        assert max(max(st["balance_rel"]) for st in ok) < 1e-8


def test_batch_rejects_single_slab_calls():
    probs = [W.random_slab(49, 20, 4, 1)]
    with oci.BatchSolver(probs) as b:
        st = oci.Stats()
        assert b.L.oci_step(b.h, st) == oci.E_STATE


def test_batch_fp32ir_matches_oracle_per_slab():
    """FP32 inner sweeps with FP64 refinement, per slab: converged flux within
    1e-10 of the FP64 oracle; sweeps within 2 (3 for J = 1) as in the single-slab
    mixed form."""
    specs = [(41, 50, 4, 1), (42, 130, 8, 1), (43, 257, 8, 2), (44, 1, 4, 1), (45, 400, 16, 1), (46, 33, 8, 2),
             (47, 128, 4, 3), (48, 77, 8, 1)]
    probs = [W.random_slab(*sp).replace(tol=1e-11) for sp in specs]
    orcs = [Oracle(p) for p in probs]
    with oci.BatchSolver(probs, precision=oci.FP32_IR) as b:
        for k in range(3):
            sts = b.step()
            for i, (p, o) in enumerate(zip(probs, orcs)):
                r = o.step(OCI)
                assert sts[i]["status"] == 0
                assert abs(sts[i]["iters"] - r["iters"]) <= (3 if p.J == 1 else 2), (i, k, sts[i]["iters"], r["iters"])
                assert rel(b.phi(i), r["phi"]) < 1e-10
                assert rel(b.psi(i), r["Psi"]) < 1e-10
                assert np.abs(b.balance(i) - r["bal"]).max() <= 1e-10 * np.abs(r["bal"]).max()


def test_batch_fp32ir_uneven_slabs_match_fp64_batch():
    """64 uneven slabs (tol 1e-10 on e): the mixed batched form converges where
    the FP64 batched form does, to the same flux within 1e-9 (both stop within
    about tol of one fixed point), and agrees with the single-slab mixed form on
    sampled slabs."""
    probs = [p.replace(max_iter=3000) for p in W.batch_of_slabs(64, j_lo=1024, j_hi=4096)]
    with oci.BatchSolver(probs) as b64:
        s64 = b64.step(allow_noconv=True)
        phi64 = {i: b64.phi(i) for i in range(len(probs)) if s64[i]["status"] == 0}
    with oci.BatchSolver(probs, precision=oci.FP32_IR) as b:
        sts = b.step(allow_noconv=True)
        for i, ph in phi64.items():
            assert sts[i]["status"] == 0, i
            assert rel(b.phi(i), ph) < 1e-9, i
            slack = 3 + 0.02 * s64[i]["iters"]  # FP32 noise in rho moves the stop on slow slabs
            assert abs(sts[i]["iters"] - s64[i]["iters"]) <= slack, (i, sts[i]["iters"], s64[i]["iters"])
        for i in (0, 21, 63):
            if i not in phi64:
                continue
            with oci.Solver(probs[i], precision=oci.FP32_IR) as s:
                st = s.step()
                assert abs(st["iters"] - sts[i]["iters"]) <= 3 + 0.02 * st["iters"]
                assert rel(b.phi(i), s.phi()) < 1e-9
        ok = [st for st in sts if st["status"] == 0]
        assert max(max(st["balance_rel"]) for st in ok) < 1e-8


@pytest.mark.parametrize("shape", ["0,32", "0,64", "2,8", "4,8", "8,8", "2,32", "4,16"])
@pytest.mark.parametrize("precision", [oci.FP64, oci.FP32_IR])
def test_batch_sweep_shapes_match_oracle(monkeypatch, shape, precision):
    """Every sweep shape the autotuner can pick (shared-memory sweep, or the
    register sweep with np angles per thread; cb cells per tile), forced through
    OCI_BATCH_SWEEP, against the FP64 oracle: sweep counts equal (FP64) or within
    2 (3 for J = 1) (FP32_IR), scalar flux within 1e-12 / 1e-10."""
    monkeypatch.setenv("OCI_BATCH_SWEEP", shape)
    specs = [(51, 70, 4, 1), (52, 131, 8, 1), (53, 66, 16, 2), (54, 1, 8, 2), (55, 90, 16, 1), (56, 45, 8, 3)]
    probs = [W.random_slab(*sp).replace(tol=1e-11) for sp in specs]
    orcs = [Oracle(p) for p in probs]
    with oci.BatchSolver(probs, precision=precision) as b:
        for k in range(2):
            sts = b.step()
            for i, (p, o) in enumerate(zip(probs, orcs)):
                r = o.step(OCI)
                assert sts[i]["status"] == 0
                if precision == oci.FP64:
                    assert sts[i]["iters"] == r["iters"], (i, k)
                    assert rel(b.phi(i), r["phi"]) < 1e-12
                else:
                    assert abs(sts[i]["iters"] - r["iters"]) <= (3 if p.J == 1 else 2), (i, k)
                    assert rel(b.phi(i), r["phi"]) < 1e-10
