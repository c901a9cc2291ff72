"""The norm entry point that allocates nothing (oci_diff_norm_noalloc).

It is meant for callers that cannot allocate device memory at the moment they
need the convergence norm; its partial sums live in a fixed device array.  This
test calls it through the C ABI on two sweeps in a row and checks each result
against the norm the regular path (oci_iterate) reports for the same sweep and
against numpy's norm of the host copies, so stale contents of the shared
scratch array would show up on the second call."""
import ctypes

import numpy as np
import pytest

from paper_2503_00264_gb300 import oci
from paper_2503_00264_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _norm_noalloc(L, a, b, out, stream):
    rc = L.oci_diff_norm_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_int64(a.numel()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream))
    return rc


def test_noalloc_norm_matches_regular_path_twice():
    import torch
    L = oci.load()
    L.oci_diff_norm_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p]
    L.oci_diff_norm_noalloc.restype = ctypes.c_int
    stream = torch.cuda.Stream()
    p = W.random_slab(71, 3000, 16, 2)
    with oci.Solver(p, stream=stream.cuda_stream) as s:
        s.set_psi(W.random_guess(p, 9))
        psis, refs = [s.psi()], []
        for _ in range(2):
            refs.append(float(s.iterate(1)[0]))
            psis.append(s.psi())
    dev = [torch.from_numpy(x).to("cuda") for x in psis]
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for k in range(2):
        assert _norm_noalloc(L, dev[k + 1], dev[k], out[k:], stream.cuda_stream) == oci.OK
    stream.synchronize()
    got = out.cpu().numpy()
    for k in range(2):
        assert abs(got[k] - refs[k]) <= 1e-12 * refs[k], (k, got[k], refs[k])
        # and against numpy's norm of the host copies of the same arrays
        host = float(np.linalg.norm((psis[k + 1] - psis[k]).ravel()))
        assert abs(got[k] - host) <= 1e-12 * host, (k, got[k], host)
    assert got[0] != got[1]


def test_noalloc_norm_rejects_too_many_values():
    import torch
    L = oci.load()
    L.oci_diff_norm_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p]
    L.oci_diff_norm_noalloc.restype = ctypes.c_int
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = L.oci_diff_norm_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                 ctypes.c_int64(33_554_433), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == oci.E_INVAL
    assert b"33,554,432" in L.oci_last_error()
