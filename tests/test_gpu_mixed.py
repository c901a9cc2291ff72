"""Mixed-precision form (FP32 inner sweeps on the correction, FP64 refinement)
against the FP64 oracle: scalar and angular flux within 1e-10 relative, balance
tallies within 1e-10 of their magnitude, sweep counts within 2 of the FP64 ones."""
import numpy as np
import pytest

from oracle import OCI, Oracle
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = [(21, 1, 4, 1), (22, 40, 8, 1), (23, 129, 16, 1), (24, 50, 8, 2), (25, 33, 4, 3)]


@pytest.mark.parametrize("seed,J,N,G", CASES)
def test_fp32_ir_matches_fp64_oracle(seed, J, N, G):
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        for k in range(3):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0
            assert abs(st["iters"] - r["iters"]) <= (3 if p.J == 1 else 2), (k, st["iters"], r["iters"])
            assert rel(s.phi(), r["phi"]) < 1e-10
            assert rel(s.psi(), r["Psi"]) < 1e-10
            assert np.abs(s.balance() - r["bal"]).max() <= 1e-10 * np.abs(r["bal"]).max()


def test_fp32_ir_sweeps_track_fp64_history():
    """Per-sweep e of the mixed form follows plain OCI's (Sec. 2.1 norm).  Late
    in a block of FP32 inner sweeps e is the difference of two FP32 corrections
    much larger than e, so its relative accuracy is about eps32 * |delta| / e
    (1e-5..1e-4 here); the converged iterate is still FP64-accurate."""
    p = W.random_slab(26, 200, 16, 1)
    guess = W.random_guess(p, 2)
    o = Oracle(p)
    o.Psi[...] = guess
    e_orc = o.iterate(60)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        s.set_psi(guess)
        e_mx = s.iterate(60)
        assert rel(s.psi(), o.Psi) < 1e-9
    keep = e_orc > 1e-6 * e_orc[0]
    assert np.all(np.abs(e_mx - e_orc)[keep] <= 1e-3 * e_orc[keep])


def test_fp32_ir_full_size_matches_fp64_path():
    """2^18-cell slab, S16 (c = 0.9, tau = 0.1), two steps: mixed vs FP64 path."""
    p = W.slab_3region(c=0.9, tau=0.1)
    with oci.Solver(p) as a, oci.Solver(p, precision=oci.FP32_IR) as b:
        for _ in range(2):
            sa, sb = a.step(), b.step()
            assert abs(sa["iters"] - sb["iters"]) <= 2
            assert max(sb["balance_rel"]) < 1e-9
        assert rel(b.phi(), a.phi()) < 1e-10
        assert rel(b.psi(), a.psi()) < 1e-10


def test_fp32_ir_noconv_keeps_last_iterate():
    p = W.random_slab(27, 60, 8, 1, c_max=0.99).replace(tol=1e-14, max_iter=5)
    o = Oracle(p)
    o.iterate(5)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        st = s.step(allow_noconv=True)
        assert st["status"] == oci.E_NOCONV
        assert rel(s.psi(), o.Psi) < 1e-6
        pp, t = s.state()
        assert t == 0.0


def _uniform_tiles(seed, J, N, G, region=128):
    """Random slab whose material and width are constant over aligned blocks of
    `region` cells (one cell type per 128-cell tile, as the tensor-core forms need)."""
    p = W.random_slab(seed, J, N, G)
    blk = np.arange(J) // region
    return p.replace(mat=(blk % p.n_mat).astype(np.int32), dx=p.dx[(blk * region) % J].copy(), tol=1e-11)


TC_CASES = [(31, 64, 8, 1), (32, 300, 16, 1), (33, 257, 8, 2), (34, 200, 16, 2), (35, 130, 4, 2)]


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
@pytest.mark.parametrize("seed,J,N,G", TC_CASES)
def test_tensor_core_forms_match_fp64_oracle(prec, seed, J, N, G):
    """Block apply on tcgen05 tensor cores (TF32, or BF16 hi/lo x3) with FP64
    refinement: flux within 1e-10 of the FP64 oracle."""
    p = _uniform_tiles(seed, J, N, G)
    o = Oracle(p)
    with oci.Solver(p, precision=prec) as s:
        for k in range(3):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0
            assert st["iters"] <= r["iters"] + 12, (st["iters"], r["iters"])
            assert rel(s.phi(), r["phi"]) < 1e-10
            assert rel(s.psi(), r["Psi"]) < 1e-10
            assert np.abs(s.balance() - r["bal"]).max() <= 1e-10 * np.abs(r["bal"]).max()


def test_tensor_core_forms_reject_mixed_tiles():
    p = W.random_slab(36, 200, 8, 1)  # a different cell type in almost every cell
    with pytest.raises(oci.OCIError) as ei:
        oci.Solver(p, precision=oci.TF32_IR)
    assert ei.value.code == oci.E_INVAL


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
def test_tensor_core_full_size_matches_fp64_path(prec):
    """Precision form of the 2^18-cell S16 slab: two steps against the FP64 path."""
    p = W.slab_3region(c=0.9, tau=0.1)
    with oci.Solver(p) as a, oci.Solver(p, precision=prec) as b:
        for _ in range(2):
            sa, sb = a.step(), b.step()
            assert sb["status"] == 0
            assert sb["iters"] <= sa["iters"] + 12
            assert max(sb["balance_rel"]) < 1e-9
        assert rel(b.phi(), a.phi()) < 1e-10
        assert rel(b.psi(), a.psi()) < 1e-10


@pytest.mark.parametrize("kernel", ["plain", "tma"])
def test_fp32_inner_kernels_both_match_oracle(kernel, monkeypatch):
    """Both FP32 inner-sweep kernels (plain, and tiles staged by 2D TMA bulk
    copies) give the FP64 oracle's answer, whichever the autotuner would pick."""
    monkeypatch.setenv("OCI_MX_INNER", kernel)
    p = W.random_slab(28, 300, 16, 2).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        info = s.info()
        assert info["inner_kernel"] == (1 if kernel == "tma" else 0)
        for k in range(2):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2
            assert rel(s.phi(), r["phi"]) < 1e-10
