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
    `region` cells (with region 128: one cell type per 128-cell tile, as the
    resident-inverse tensor-core kernels need)."""
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


@pytest.mark.parametrize("pipe", ["1", "0"])
@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
@pytest.mark.parametrize("seed,J,N,G", [(37, 300, 16, 1), (38, 257, 8, 2)])
def test_tensor_core_resident_inverse_kernels_match_oracle(pipe, prec, seed, J, N, G, monkeypatch):
    """The two tensor-core kernels that keep the inverse resident in shared
    memory (4NG <= 128; persistent, and one tile per CTA) against the FP64
    oracle, as the streamed kernel is above."""
    monkeypatch.setenv("OCI_TC_BIG", "0")
    monkeypatch.setenv("OCI_TC_PIPE", pipe)
    p = _uniform_tiles(seed, J, N, G)
    o = Oracle(p)
    with oci.Solver(p, precision=prec) as s:
        for k in range(2):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0
            assert st["iters"] <= r["iters"] + 12, (st["iters"], r["iters"])
            assert rel(s.phi(), r["phi"]) < 1e-10
            assert rel(s.psi(), r["Psi"]) < 1e-10


def test_tensor_core_forms_reject_mixed_tiles(monkeypatch):
    """A different cell type in almost every cell would need a pass per cell over
    each tile: rejected.  Region boundaries inside tiles are taken by the streamed
    kernel but not by the resident-inverse kernels (test hook)."""
    p = W.random_slab(36, 200, 8, 1)
    with pytest.raises(oci.OCIError) as ei:
        oci.Solver(p, precision=oci.TF32_IR)
    assert ei.value.code == oci.E_INVAL
    monkeypatch.setenv("OCI_TC_BIG", "0")
    with pytest.raises(oci.OCIError) as ei:
        oci.Solver(_uniform_tiles(39, 300, 8, 1, region=100), precision=oci.TF32_IR)
    assert ei.value.code == oci.E_INVAL


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
@pytest.mark.parametrize("seed,J,N,G,region", [(46, 500, 16, 1, 100), (47, 700, 16, 3, 180), (48, 333, 16, 8, 100),
                                               (49, 129, 8, 2, 100)])
def test_tensor_core_forms_with_regions_inside_tiles_match_oracle(prec, seed, J, N, G, region):
    """Region boundaries that fall inside 128-cell tiles (regions of 100 and 180
    cells): the streamed kernel takes such a tile once per cell type in it and
    keeps each pass's cells; flux within 1e-10 of the FP64 oracle over three steps
    at 64, 192, 512 and 32 unknowns per cell."""
    p = _uniform_tiles(seed, J, N, G, region=region)
    o = Oracle(p)
    with oci.Solver(p, precision=prec) as s:
        for k in range(3):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0
            assert st["iters"] <= r["iters"] + 12, (st["iters"], r["iters"])
            assert rel(s.phi(), r["phi"]) < 1e-10
            assert rel(s.psi(), r["Psi"]) < 1e-10


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
@pytest.mark.parametrize("N,J", [(16, 2 ** 18), (8, 2 ** 17)])
def test_tensor_core_full_size_matches_fp64_path(prec, N, J):
    """Precision form of the three-region slab at full size (2^18 cells at S16;
    2^17 at S8, 32 unknowns per cell: two K-chunks per tile in the full form, one
    in the coupling form, and more than four tiles per CTA): two steps against
    the FP64 path."""
    p = W.slab_3region(c=0.9, tau=0.1, J=J, N=N)
    with oci.Solver(p) as a, oci.Solver(p, precision=prec) as b:
        for _ in range(2):
            sa, sb = a.step(), b.step()
            assert sb["status"] == 0
            assert sb["iters"] <= sa["iters"] + 12
            assert max(sb["balance_rel"]) < 1e-9
        assert rel(b.phi(), a.phi()) < 1e-10
        assert rel(b.psi(), a.psi()) < 1e-10


@pytest.mark.parametrize("kernel", ["plain", "tma", "reg", "tiled", "tiledp", "tiledb", "two"])
def test_fp32_inner_kernels_all_match_oracle(kernel, monkeypatch):
    """Every FP32 inner-sweep kernel (plain, tiles staged by 2D TMA bulk copies,
    angles split over threads with t in registers, and that on tile-major
    correction arrays, one tile per block, persistent, or persistent with the
    tiles moved by 1D bulk copies) gives the FP64 oracle's answer, whichever the
    autotuner would pick."""
    monkeypatch.setenv("OCI_MX_INNER", kernel)
    p = W.random_slab(28, 300, 16, 2).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        info = s.info()
        assert info["inner_kernel"] == {"plain": 0, "tma": 1, "reg": 3, "tiled": 4, "tiledp": 5,
                                        "tiledb": 6, "two": 9}[kernel]
        for k in range(2):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2
            assert rel(s.phi(), r["phi"]) < 1e-10


@pytest.mark.parametrize("kernel,shape", [("reg", "32,8"), ("reg", "64,4"), ("reg", "128,2"), ("reg", "64,2"),
                                          ("tiled", "32,8"), ("tiled", "64,4"), ("tiled", "64,2"),
                                          ("tiled", "32,2"), ("tiledp", "32,8"), ("tiledp", "64,4"),
                                          ("tiledp", "64,2"), ("tiledp", "128,2"), ("tiledb", "32,8"),
                                          ("tiledb", "64,4"),
                                          ("tiledb", "64,2"), ("tiledb", "32,2"), ("two", "32,8"),
                                          ("two", "32,4"), ("two", "64,4"), ("twoocc", "32,8"),
                                          ("twoocc", "32,4"), ("twoocc", "64,4")])
def test_fp32_register_inner_shapes_match_oracle(kernel, shape, monkeypatch):
    """Register FP32 inner sweeps (row layout, and tile-major with T = 32 or 64
    cells) at each angle split (P = 8, 4, 2 chunks of S16 angles, G = 1) on a
    ragged slab (J = 333: a partial last tile): flux within 1e-10 of the oracle."""
    monkeypatch.setenv("OCI_MX_INNER", kernel)
    monkeypatch.setenv("OCI_SWEEP_SHAPE", shape)
    p = W.random_slab(29, 333, 16, 1).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        info = s.info()
        cb, P = (int(x) for x in shape.split(","))
        assert (info["inner_kernel"], info["cells_per_block"], info["angle_chunks"]) == (
            {"reg": 3, "tiled": 4, "tiledp": 5, "tiledb": 6, "two": 9, "twoocc": 10}[kernel], cb, P)
        for k in range(2):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2
            assert rel(s.phi(), r["phi"]) < 1e-10


def test_fp32_multi_sweep_launch_matches_single_sweep(monkeypatch):
    """In the graph the persistent tiled FP32 sweep runs several sweeps per
    cooperative launch (grid barrier per sweep, refinement under an IF node);
    the same steps with one sweep per launch give the same sweep counts and the
    same iterate (per-tile arithmetic is identical; only the order in which
    block partials of the norm are formed may differ)."""
    monkeypatch.setenv("OCI_MX_INNER", "tiledp")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", "64,4")
    p = W.random_slab(31, 5000, 16, 1).replace(tol=1e-11)
    res = {}
    for multi in ("1", "0"):
        monkeypatch.setenv("OCI_MX_MULTI", multi)
        with oci.Solver(p, precision=oci.FP32_IR) as s:
            its = [s.step()["iters"] for _ in range(3)]
            res[multi] = (its, s.psi(), s.phi())
    assert res["1"][0] == res["0"][0]
    assert rel(res["1"][1], res["0"][1]) < 1e-13
    o = Oracle(p)
    for k in range(3):
        r = o.step(OCI)
        assert abs(res["1"][0][k] - r["iters"]) <= 2
    assert rel(res["1"][2], r["phi"]) < 1e-10


@pytest.mark.parametrize("kernel,J,shape", [("two", 5000, "64,4"), ("two", 40000, "64,4"), ("two", 40000, "32,8"),
                                            ("two", 333, "32,4"), ("two", 64, "32,8"), ("twoocc", 40000, "32,4"),
                                            ("twoocc", 5000, "32,8"), ("warp", 40000, "32,4"),
                                            ("warp", 5000, "32,4"), ("warp", 333, "32,4"), ("warp", 64, "32,4"),
                                            ("warp", 40, "32,4")])
def test_fp32_two_sweep_passes_equal_one_sweep_launches(kernel, J, shape, monkeypatch):
    """Two inner sweeps per pass (each block walks a run of tiles, the second
    sweep's inflows from the first sweep's values held in shared memory, the
    run's two outside neighbours recomputed by the block) give bit for bit the
    iterates, norms and sweep counts of one sweep per launch of the same
    kernel (default and high-occupancy builds): the cell arithmetic and the
    order of every sum are the same.  Runs
    of one tile (J = 5000: 79 tiles, one per block), of several tiles, a
    partial last tile, and a one-block slab; the first sweep of a pass ending
    an inner block (refinement or stop) takes the recompute path.  The
    warp-run kernel (each warp walks its own run of 8-cell groups, inflows
    of the second sweep from a per-warp ring) the same way: runs of 1 to 14
    groups, warps with empty runs (a 40-cell slab)."""
    monkeypatch.setenv("OCI_MX_INNER", kernel)
    monkeypatch.setenv("OCI_SWEEP_SHAPE", shape)
    p = W.random_slab(33, J, 16, 1).replace(tol=1e-11)
    res = {}
    for multi in ("1", "0"):
        monkeypatch.setenv("OCI_MX_MULTI", multi)
        with oci.Solver(p, precision=oci.FP32_IR) as s:
            assert s.info()["inner_kernel"] == {"two": 9, "twoocc": 10, "warp": 12}[kernel]
            sts = [s.step() for _ in range(3)]
            res[multi] = ([(t["iters"], t["refinements"], t["e"]) for t in sts], s.psi(), s.phi())
    assert res["1"][0] == res["0"][0]
    assert np.array_equal(res["1"][1], res["0"][1])
    o = Oracle(p)
    for k in range(3):
        r = o.step(OCI)
        assert abs(res["1"][0][k][0] - r["iters"]) <= 2
    assert rel(res["1"][2], r["phi"]) < 1e-10


@pytest.mark.parametrize("seed,J,N", [(97, 1000, 8), (98, 257, 8), (99, 1000, 32), (100, 70, 32), (101, 17, 16),
                                      (102, 20000, 8), (103, 9000, 32)])
def test_fp32_warp_run_kernel_angle_counts(seed, J, N, monkeypatch):
    """The warp-run two-sweep kernel at S8 (16 cells per warp step, two lanes
    per cell) and S32 (4 cells, eight lanes): sweep counts within 2 of the
    FP64 oracle's and flux within 1e-10 of it, on ragged slabs."""
    monkeypatch.setenv("OCI_MX_INNER", "warp")
    p = W.random_slab(seed, J, N, 1).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        info = s.info()
        assert (info["inner_kernel"], info["cells_per_block"], info["angle_chunks"]) == (12, 32, N // 4)
        for k in range(3):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2, (st["iters"], r["iters"])
            assert rel(s.phi(), r["phi"]) < 1e-10
            assert rel(s.psi(), r["Psi"]) < 1e-10


@pytest.mark.parametrize("seed,J,N,G", [(91, 1, 4, 1), (92, 33, 4, 2), (93, 257, 8, 1), (94, 129, 8, 4),
                                        (95, 100, 4, 1), (96, 1000, 32, 1)])
def test_fp32_two_sweep_passes_small_and_multigroup(seed, J, N, G, monkeypatch):
    """Two sweeps per pass on one-cell and partial-tile slabs, few angles and
    several groups: the sweep counts of the one-sweep persistent kernel and flux
    within 1e-10 of the FP64 oracle.  Sweeps are within 2 of the oracle's, but
    for one cell: there plain OCI is exact after one sweep, while each FP32
    inner block resolves only about 7 digits, so the mixed form needs a
    refinement sweep per 7 digits (3 extra at tol 1e-11)."""
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    res = {}
    for kern in ("two", "tiledp"):
        monkeypatch.setenv("OCI_MX_INNER", kern)
        with oci.Solver(p, precision=oci.FP32_IR) as s:
            assert s.info()["inner_kernel"] == {"two": 9, "tiledp": 5}[kern]
            res[kern] = [(s.step(), s.phi()) for _ in range(2)]
    o = Oracle(p)
    for k in range(2):
        r = o.step(OCI)
        st, phi = res["two"][k]
        assert st["status"] == 0 and st["iters"] == res["tiledp"][k][0]["iters"]
        assert abs(st["iters"] - r["iters"]) <= (3 if J == 1 else 2)
        assert rel(phi, r["phi"]) < 1e-10


RB_CASES = [(71, 33, 8, 1, None), (72, 129, 8, 2, None), (73, 1, 4, 1, None), (74, 300, 16, 1, None),
            (75, 257, 16, 1, "32,4"), (76, 300, 16, 1, "64,2"), (77, 95, 4, 2, "32,2"), (78, 5000, 16, 1, "64,4"),
            (79, 65, 16, 1, "32,8")]


@pytest.mark.parametrize("kernel", ["1", "2"])
@pytest.mark.parametrize("seed,J,N,G,shape", RB_CASES)
def test_fp32_red_black_matches_oracle(seed, J, N, G, shape, kernel, monkeypatch):
    """Red-black ordering of the mixed form (even cells then odd cells per
    inner sweep, colour-ordered tile-major layout; kernel 1: one sweep per pass,
    in place, grid barrier between the colours; kernel 2: two sweeps per pass
    over the correction, each block walking a run of tiles) against the
    oracle's FP64 red-black sweep: sweep counts within 2 (3 for J = 1), flux
    within 1e-10; forced shapes cover both tile widths, one-tile runs
    (J = 5000 at 64-cell tiles) and an odd partial last tile."""
    from oracle import RB
    if kernel == "2" and shape == "64,2":
        pytest.skip("two sweeps per pass keep at most 4 angles per thread")
    monkeypatch.setenv("OCI_MX_RB", kernel)
    if shape:
        monkeypatch.setenv("OCI_SWEEP_SHAPE", shape)
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        s.set_ordering(oci.ORDER_RED_BLACK)
        info = s.info()
        assert info["inner_kernel"] == {"1": 7, "2": 11}[kernel]
        if shape:
            assert (info["cells_per_block"], info["angle_chunks"]) == tuple(int(x) for x in shape.split(","))
        for k in range(2):
            r = o.step(RB)
            st = s.step()
            assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= (3 if J == 1 else 2), (st["iters"], r["iters"])
            assert rel(s.phi(), r["phi"]) < 1e-10
            assert rel(s.psi(), r["Psi"]) < 1e-10
        s.set_ordering(oci.ORDER_JACOBI)  # back to the tuned Jacobi inner sweep
        assert s.info()["inner_kernel"] not in (7, 11)
        r = o.step(OCI)
        st = s.step()
        assert abs(st["iters"] - r["iters"]) <= 2 and rel(s.phi(), r["phi"]) < 1e-10


@pytest.mark.parametrize("J,shape", [(40000, "32,8"), (40000, "64,4"), (5000, "32,4"), (333, "64,8"), (65, "32,4")])
def test_fp32_red_black_two_sweep_passes_equal_one_sweep_launches(J, shape, monkeypatch):
    """Red-black sweeps two per pass (graph) and one per launch (host-driven)
    of the same kernel give the same iterates bit for bit, the same norms and
    sweep counts: the cell arithmetic and the order of every sum agree."""
    monkeypatch.setenv("OCI_MX_RB", "2")
    monkeypatch.setenv("OCI_SWEEP_SHAPE", shape)
    p = W.random_slab(34, J, 16, 1).replace(tol=1e-11)
    res = {}
    for multi in ("1", "0"):
        monkeypatch.setenv("OCI_MX_MULTI", multi)
        with oci.Solver(p, precision=oci.FP32_IR) as s:
            s.set_ordering(oci.ORDER_RED_BLACK)
            assert s.info()["inner_kernel"] == 11
            sts = [s.step() for _ in range(3)]
            res[multi] = ([(t["iters"], t["refinements"], t["e"]) for t in sts], s.psi())
    assert res["1"][0] == res["0"][0]
    assert np.array_equal(res["1"][1], res["0"][1])


def test_fp32_red_black_full_size_fewer_sweeps_same_answer():
    """2^18-cell slab (c = 0.9, tau = 0.1): the red-black mixed form converges in
    well under 0.7x the Jacobi sweeps to the FP64 red-black answer."""
    p = W.slab_3region(c=0.9, tau=0.1)
    with oci.Solver(p) as a, oci.Solver(p, precision=oci.FP32_IR) as b:
        a.set_ordering(oci.ORDER_RED_BLACK)
        b.set_ordering(oci.ORDER_RED_BLACK)
        sa, sb = a.step(), b.step()
        assert abs(sb["iters"] - sa["iters"]) <= 2
        assert rel(b.phi(), a.phi()) < 1e-10


@pytest.mark.parametrize("seed,J,N,G", [(81, 40, 128, 1), (82, 37, 8, 16), (83, 70, 32, 4)])
@pytest.mark.parametrize("ordering", ["jacobi", "rb"])
def test_fp32_ir_max_sizes(seed, J, N, G, ordering):
    """The mixed form at the size limits (N = 128; G = 16; N*G = 128), in both
    orderings: whichever inner kernels fit these shapes (per-type tables staged
    in shared memory or read from global memory) give the oracle's answer."""
    from oracle import RB
    p = W.random_slab(seed, J, N, G).replace(tol=1e-10)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        if ordering == "rb":
            s.set_ordering(oci.ORDER_RED_BLACK)
        r = o.step(RB if ordering == "rb" else OCI)
        st = s.step()
        assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2, (st["iters"], r["iters"])
        assert rel(s.phi(), r["phi"]) < 1e-9


@pytest.mark.parametrize("kernel,kind", [("tiledp", 5), ("reg", 3)])
def test_fp32_multigroup_16_cell_tiles_match_oracle(kernel, kind, monkeypatch):
    """G = 8, S16: the FP32 inner sweeps with 16-cell tiles (8 angles per thread,
    2 chunks x 8 groups x 16 cells = 256 threads), which the autotuner offers
    for many groups, against the oracle (ragged J: a partial last tile)."""
    monkeypatch.setenv("OCI_MX_INNER", kernel)
    monkeypatch.setenv("OCI_SWEEP_SHAPE", "16,2")
    p = W.random_slab(101, 203, 16, 8).replace(tol=1e-10)
    o = Oracle(p)
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        info = s.info()
        assert (info["inner_kernel"], info["cells_per_block"], info["angle_chunks"]) == (kind, 16, 2)
        for k in range(2):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0 and abs(st["iters"] - r["iters"]) <= 2
            assert rel(s.phi(), r["phi"]) < 1e-10


# more than 128 unknowns per cell: A^{-1} in M-tiles of 128 rows, streamed in K-chunks of 32
TC_BIG_CASES = [(41, 300, 16, 3), (42, 257, 16, 4), (43, 200, 10, 4), (44, 140, 32, 4), (45, 129, 16, 8)]


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
@pytest.mark.parametrize("seed,J,N,G", TC_BIG_CASES)
def test_tensor_core_forms_more_than_128_unknowns_match_oracle(prec, seed, J, N, G):
    """4NG = 192 (one N-tile narrower than 256), 256, 160 (ten K-chunks of 16),
    512 (two N-tiles of 256): flux within 1e-10 of the FP64 oracle over three
    steps, ragged last tile."""
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


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
def test_tensor_core_multigroup_recipe_matches_oracle_per_group(prec):
    """The 8-group, S16, 4-material recipe (512 unknowns per cell, blocks of
    256 cells) on 1024 cells: two converged steps against the oracle, per group
    within 1e-8 of each group's scale and 1e-10 of the largest."""
    p = W.slab_multigroup(J=1024, region=256)
    o = Oracle(p, share_factors=True)
    with oci.Solver(p, precision=prec) as s:
        for k in range(2):
            r = o.step(OCI)
            st = s.step()
            assert st["status"] == 0
            assert st["iters"] <= r["iters"] + 12, (st["iters"], r["iters"])
            phi = s.phi()
            assert rel(phi, r["phi"]) < 1e-10
            d = np.abs(phi - r["phi"]).max(axis=(0, 2)) / np.abs(r["phi"]).max(axis=(0, 2))
            assert d.max() < 1e-8, d


@pytest.mark.parametrize("prec", [oci.TF32_IR, oci.BF16X3_IR])
@pytest.mark.parametrize("seed,J,N,G,region", [(50, 700, 16, 1, 128), (51, 333, 8, 2, 100), (52, 257, 16, 4, 128),
                                               (53, 200, 10, 4, 128), (54, 40, 8, 1, 128), (55, 300, 16, 8, 100),
                                               (56, 140, 32, 4, 128)])
def test_tensor_core_coupling_sweeps_equal_full_sweeps(prec, seed, J, N, G, region, monkeypatch):
    """Inner sweeps after the first of a refinement block as delta = z + (A~^{-1} B) u
    over the n/2 inflow columns (z = A~^{-1} r from the block's first sweep) against
    every sweep as the full A~^{-1} (r + B delta) (test hook OCI_TC_HALF=0): the same
    converged step within 1e-10 of each other and of the oracle, sweeps within 12;
    64, 128, 256, 160 and 512 unknowns per cell (above 256 the old correction comes
    from HBM), region boundaries inside tiles, one tile."""
    p = _uniform_tiles(seed, J, N, G, region=region)
    o = Oracle(p)
    ref = [o.step(OCI) for _ in range(2)]
    out = {}
    for half in ("1", "0"):
        monkeypatch.setenv("OCI_TC_HALF", half)
        with oci.Solver(p, precision=prec) as s:
            sts = [s.step() for _ in range(2)]
            out[half] = (sts, s.phi(), s.psi())
    for half in ("1", "0"):
        sts, phi, psi = out[half]
        for k in range(2):
            assert sts[k]["status"] == 0
            assert sts[k]["iters"] <= ref[k]["iters"] + 12, (half, k, sts[k]["iters"], ref[k]["iters"])
        assert rel(phi, ref[-1]["phi"]) < 1e-10
        assert rel(psi, o.Psi) < 1e-10
    assert rel(out["1"][1], out["0"][1]) < 1e-10
