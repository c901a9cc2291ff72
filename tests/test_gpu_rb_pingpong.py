"""FP64 red-black sweeps with ping-pong buffers (both colours read Psi[cur] and
write Psi[cur^1], the second colour taking its neighbours' new values from
Psi[cur^1]; the default) against the same half sweeps in place on Psi[cur]
(OCI_RB_FP64=inplace).  Every cell reads the same values and every block sums
the same partials, so steps, exact-count iterations, norm history, iterates and
flux agree bit for bit; the sweep counts equal the oracle's red-black sweep; a
step that does not converge leaves the last iterate readable and commits
nothing."""
import numpy as np
import pytest

from oracle import RB, Oracle
from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _layout(monkeypatch, inplace):
    monkeypatch.setenv("OCI_AUTOTUNE", "0")  # the same launch shape in both runs
    if inplace:
        monkeypatch.setenv("OCI_RB_FP64", "inplace")
    else:
        monkeypatch.delenv("OCI_RB_FP64", raising=False)


def _solve(p, monkeypatch, inplace):
    _layout(monkeypatch, inplace)
    with oci.Solver(p) as s:
        s.set_ordering(oci.ORDER_RED_BLACK)
        sts = [s.step() for _ in range(2)]
        eh = s.e_hist().copy()
        it = s.iterate(5)
        return ([(t["status"], t["iters"], t["e"], t["rho"]) for t in sts], eh, it, s.psi(), s.phi())


@pytest.mark.parametrize("seed,J,N,G", [(141, 1, 4, 1), (142, 2, 4, 1), (143, 33, 8, 1), (144, 257, 8, 2),
                                        (145, 1000, 16, 1), (146, 4097, 8, 3)])
def test_ping_pong_equals_in_place_bitwise(seed, J, N, G, monkeypatch):
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    a = _solve(p, monkeypatch, inplace=False)
    b = _solve(p, monkeypatch, inplace=True)
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    o = Oracle(p)
    for k in range(2):
        r = o.step(RB)
        assert a[0][k][0] == 0 and a[0][k][1] == r["iters"], (k, a[0][k], r["iters"])


def test_ping_pong_noconv_keeps_state_and_last_iterate(monkeypatch):
    p = W.random_slab(147, 301, 8, 1, c_max=0.99).replace(tol=1e-15, max_iter=4)
    out = {}
    for inplace in (False, True):
        _layout(monkeypatch, inplace)
        with oci.Solver(p) as s:
            s.set_ordering(oci.ORDER_RED_BLACK)
            pp0, t0 = s.state()
            with pytest.raises(oci.OCIError) as ei:
                s.step()
            assert ei.value.code == oci.E_NOCONV
            pp1, t1 = s.state()
            assert t1 == t0 and np.array_equal(pp0, pp1)
            out[inplace] = s.psi()
    assert np.any(out[False])
    assert np.array_equal(out[False], out[True])


def _legal(shape, N, G):
    kind, cb, P = shape.split(",")
    cb, P = int(cb), int(P)
    thr = cb * G * P
    if kind == "s":
        return N % P == 0 and 32 <= thr <= 256 and cb * (G * N * 4 + G * P * 4) * 8 + 512 <= 100 * 1024
    return N % P == 0 and N // P in (2, 4, 8) and cb in (16, 32, 64) and thr <= 256 and thr % 32 == 0 and thr >= 64


@pytest.mark.parametrize("shape", ["s,32,1", "s,64,2", "s,128,1", "r,16,4", "r,32,2", "r,64,1", "r,16,2"])
@pytest.mark.parametrize("seed,J,N,G", [(151, 1, 4, 1), (152, 77, 8, 1), (153, 300, 8, 2), (154, 1025, 16, 1)])
def test_forced_red_black_shapes_match_oracle(shape, seed, J, N, G, monkeypatch):
    """Every red-black form the setup tuner can pick (staged or register, ping-pong),
    forced with OCI_RB_SHAPE: the oracle's red-black sweep counts, flux within 1e-12."""
    if not _legal(shape, N, G):
        pytest.skip("shape not legal for this N, G")
    monkeypatch.setenv("OCI_RB_SHAPE", shape)
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p) as s:
        s.set_ordering(oci.ORDER_RED_BLACK)
        info = s.info()
        assert info["sweep_kernel"] == (3 if shape[0] == "r" else 2)
        assert (info["cells_per_block"], info["angle_chunks"]) == tuple(int(x) for x in shape.split(",")[1:])
        for k in range(2):
            r = o.step(RB)
            st = s.step()
            assert st["status"] == 0 and st["iters"] == r["iters"], (k, st["iters"], r["iters"])
            assert float(np.abs(s.phi() - r["phi"]).max() / np.abs(r["phi"]).max()) < 1e-12
            assert float(np.abs(s.psi() - r["Psi"]).max() / np.abs(r["Psi"]).max()) < 1e-11


def test_illegal_red_black_shape_rejected(monkeypatch):
    monkeypatch.setenv("OCI_RB_SHAPE", "r,16,3")
    with oci.Solver(W.random_slab(155, 40, 8, 1)) as s:
        with pytest.raises(oci.OCIError) as ei:
            s.set_ordering(oci.ORDER_RED_BLACK)
        assert ei.value.code == oci.E_INVAL
        assert s.info()["sweep_kernel"] in (0, 1)  # still Jacobi
        assert s.step()["status"] == 0


def test_switching_ordering_between_steps_keeps_the_state():
    """Jacobi, red-black, red-black, Jacobi steps on one handle: each step starts
    from the previous step's state (the red-black shapes are timed at the first
    switch without touching it) and matches the oracle's sequence of the same
    orderings."""
    from oracle import OCI
    p = W.random_slab(156, 500, 8, 2).replace(tol=1e-11)
    o = Oracle(p)
    with oci.Solver(p) as s:
        for order in (OCI, RB, RB, OCI):
            s.set_ordering(oci.ORDER_RED_BLACK if order == RB else oci.ORDER_JACOBI)
            r = o.step(order)
            st = s.step()
            assert st["status"] == 0 and st["iters"] == r["iters"], (order, st["iters"], r["iters"])
            assert float(np.abs(s.phi() - r["phi"]).max() / np.abs(r["phi"]).max()) < 1e-12


def test_first_switch_to_red_black_keeps_the_last_iterate():
    """The red-black shapes are timed on the first switch: an unconverged step's
    last iterate, the carried state and the time are untouched by it, and the
    next (red-black) step starts from that iterate as the oracle's does."""
    p = W.random_slab(157, 3000, 8, 1, c_max=0.99).replace(tol=1e-14, max_iter=6)
    with oci.Solver(p) as s:
        with pytest.raises(oci.OCIError) as ei:
            s.step()
        assert ei.value.code == oci.E_NOCONV
        psi0 = s.psi()
        pp0, t0 = s.state()
        s.set_ordering(oci.ORDER_RED_BLACK)
        assert s.info()["tuned_sweep_us"] > 0
        assert np.array_equal(s.psi(), psi0)
        pp1, t1 = s.state()
        assert t1 == t0 and np.array_equal(pp0, pp1)
