"""The FP64 refinement of the mixed forms converts between the FP32 correction
or residual and FP64 on the integer pipe and reads an upstream neighbour inside
its tile back from the refined iterate; with OCI_MX_OUTER_CVT=hw it uses the
compiler's conversions and recomputes every neighbour.  Both give the same
bits: iterates, flux, norm history and sweep and refinement counts, for the
FP32, TF32 and split-BF16 inner solves, Jacobi and red-black order, ragged and
multigroup slabs, the batched form, and slabs whose residuals are exactly zero
or fall below the binary32 normal range (the conversions' fallback paths).
The inner kernel and its shape are fixed (no timing-based choice), so that the
two runs differ only in the refinement."""
import numpy as np
import pytest

from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(p, precision, monkeypatch, hw, red_black=False, steps=3, rb_shape="32,4"):
    monkeypatch.setenv("OCI_AUTOTUNE", "0")
    monkeypatch.setenv("OCI_MX_RB", "2")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", rb_shape)
    if hw:
        monkeypatch.setenv("OCI_MX_OUTER_CVT", "hw")
    else:
        monkeypatch.delenv("OCI_MX_OUTER_CVT", raising=False)
    with oci.Solver(p, precision=precision) as s:
        if red_black:
            s.set_ordering(oci.ORDER_RED_BLACK)
        sts = [s.step(allow_noconv=True) for _ in range(steps)]
        return ([(t["status"], t["iters"], t["refinements"], t["e"]) for t in sts], s.psi(), s.phi())


CASES = [
    (oci.FP32_IR, 101, 5000, 16, 1, False),
    (oci.FP32_IR, 102, 333, 8, 2, False),
    (oci.FP32_IR, 103, 1, 4, 1, False),
    (oci.FP32_IR, 104, 2049, 16, 1, "32,4"),
    (oci.FP32_IR, 105, 700, 8, 2, "32,2"),
    (oci.TF32_IR, 106, 3000, 16, 1, False),
    (oci.BF16X3_IR, 107, 1000, 8, 2, False),
]


@pytest.mark.parametrize("precision,seed,J,N,G,rb", CASES)
def test_integer_conversions_give_the_same_bits(precision, seed, J, N, G, rb, monkeypatch):
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    if precision != oci.FP32_IR:  # the tensor-core forms take one cell type per 128-cell tile
        blk = np.arange(J) // 128
        p = p.replace(mat=(blk % p.n_mat).astype(np.int32), dx=p.dx[(blk * 128) % J].copy())
    a = _run(p, precision, monkeypatch, hw=False, red_black=bool(rb), rb_shape=rb or "32,4")
    b = _run(p, precision, monkeypatch, hw=True, red_black=bool(rb), rb_shape=rb or "32,4")
    assert a[0] == b[0]
    assert all(st[0] == 0 for st in a[0])
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("scale", [0.0, 1e-36, 1e17])
def test_zero_and_extreme_residuals_give_the_same_bits(scale, monkeypatch):
    """scale 0: no source, no inflow, zero initial flux (every residual exactly
    zero); 1e-36: residuals in and below the binary32 subnormal range; 1e17:
    large residuals whose FP32 squares in the norm still stay finite.  The solves
    need not converge (FP32 cannot hold the tiny corrections); both conversion
    paths must agree."""
    p = W.random_slab(111, 700, 8, 1)
    p = p.replace(Q=p.Q * scale, psi_init=p.psi_init * scale, inc_left=p.inc_left * scale,
                  inc_right=p.inc_right * scale, tol=1e-11 * max(scale, 1e-300), max_iter=300)
    a = _run(p, oci.FP32_IR, monkeypatch, hw=False, steps=2)
    b = _run(p, oci.FP32_IR, monkeypatch, hw=True, steps=2)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    if scale == 0.0:
        assert not np.any(a[1])


def test_batched_refinement_gives_the_same_bits(monkeypatch):
    specs = [(121, 50, 4, 1), (122, 130, 8, 1), (123, 257, 8, 2), (124, 1, 4, 1), (125, 400, 16, 1),
             (126, 128, 4, 3)]
    probs = [W.random_slab(*sp).replace(tol=1e-11) for sp in specs]
    out = {}
    monkeypatch.setenv("OCI_AUTOTUNE", "0")
    for hw in (False, True):
        if hw:
            monkeypatch.setenv("OCI_MX_OUTER_CVT", "hw")
        else:
            monkeypatch.delenv("OCI_MX_OUTER_CVT", raising=False)
        with oci.BatchSolver(probs, precision=oci.FP32_IR) as b:
            sts = [b.step() for _ in range(2)]
            out[hw] = ([[(s["status"], s["iters"]) for s in st] for st in sts],
                       [b.psi(i) for i in range(len(probs))])
    assert out[False][0] == out[True][0]
    for x, y in zip(out[False][1], out[True][1]):
        assert np.array_equal(x, y)
