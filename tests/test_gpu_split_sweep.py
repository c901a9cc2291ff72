"""One OCI sweep in two calls (oci_iterate_part): the blocks that read no
incident flux first, then the first and the last block with e of the whole
sweep.  A subdomain of a decomposed slab (Sec. 4) sweeps its interior that way
while its neighbours' edge values are in flight.  The two calls must be one
oci_iterate sweep bit for bit -- same cells, same block partials, same
fixed-order sum -- also when the incident fluxes change between them, for the
staged and the register form of the FP64 sweep and for one, two, three and
many blocks, and after the state (psi_{k-1/2}) changes between sweeps."""
import numpy as np
import pytest

from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (seed, J, N, G, OCI_SWEEP_REG, OCI_SWEEP_SHAPE): blocks of 64 or 32 cells
CASES = [(61, 3000, 16, 1, "0", "64,2"), (62, 3000, 16, 1, "1", "64,4"), (63, 40, 8, 1, "0", "64,2"),
         (64, 100, 8, 2, "0", "64,2"), (65, 150, 16, 1, "1", "64,4"), (66, 333, 8, 2, "1", "32,2"),
         (67, 2049, 32, 1, "1", "32,4")]


@pytest.mark.parametrize("seed,J,N,G,reg,shape", CASES)
def test_split_sweep_equals_one_sweep(seed, J, N, G, reg, shape, monkeypatch):
    monkeypatch.setenv("OCI_SWEEP_REG", reg)
    monkeypatch.setenv("OCI_SWEEP_SHAPE", shape)
    p = W.random_slab(seed, J, N, G)
    psi0 = W.random_guess(p, 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    with oci.Solver(p) as a, oci.Solver(p) as b:
        ia, ib = a.info(), b.info()
        assert (ia["sweep_kernel"], ia["cells_per_block"]) == (ib["sweep_kernel"], ib["cells_per_block"])
        assert ia["sweep_kernel"] == int(reg)
        a.set_psi(psi0)
        b.set_psi(psi0)
        for k in range(6):
            if k >= 2:  # new incident fluxes: before the sweep, or between its two parts
                il, ir = rng.uniform(0.0, 2.0, (G, N, 2)), rng.uniform(0.0, 2.0, (G, N, 2))
                a.set_boundary(il, ir)
            if k == 4:  # a new psi_{k-1/2}: the split sweep recomputes its step constant
                pp = rng.uniform(0.0, 1.0, (J, G, N, 2))
                a.set_state(pp, 0.5)
                b.set_state(pp, 0.5)
            ea = a.iterate(1)
            eb = np.zeros(1)
            b.iterate_part(0)
            if k >= 2:
                b.set_boundary(il, ir)
            b.iterate_part(1, eb)
            assert ea[0] == eb[0], (k, ea[0], eb[0])
            assert np.array_equal(a.psi(), b.psi())


def test_split_sweep_rejects_misuse():
    p = W.random_slab(68, 500, 8, 1)
    with oci.Solver(p) as s:
        with pytest.raises(oci.OCIError) as ei:
            s.iterate_part(1)
        assert ei.value.code == oci.E_STATE
        s.iterate_part(0)
        for call in (lambda: s.iterate_part(0), lambda: s.iterate(1), lambda: s.step()):
            with pytest.raises(oci.OCIError) as ei:
                call()
            assert ei.value.code == oci.E_STATE
        s.iterate_part(1)  # the pending sweep still completes
        s.set_ordering(oci.ORDER_RED_BLACK)
        with pytest.raises(oci.OCIError) as ei:
            s.iterate_part(0)
        assert ei.value.code == oci.E_STATE
    with oci.Solver(p, precision=oci.FP32_IR) as s:
        with pytest.raises(oci.OCIError) as ei:
            s.iterate_part(0)
        assert ei.value.code == oci.E_STATE
