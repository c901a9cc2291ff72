"""C-ABI library checks that need no GPU: it builds for sm_103a, loads, exports
every function include/oci.h declares, and rejects invalid problems with
OCI_E_INVAL before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2503_00264_gb300 import build, oci
from paper_2503_00264_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return oci.load()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "oci.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(\w+)\s*\(", hdr, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(oci.EXPORTS)


def test_struct_layouts_match_the_compiled_header(tmp_path):
    """sizeof and every field offset of oci_problem, oci_stats and oci_info as a C
    compiler lays them out from include/oci.h equal those of the ctypes binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"oci_problem": oci.Problem, "oci_stats": oci.Stats, "oci_info": oci.Info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "oci.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_struct_layout_matches_header():
    # oci_problem: 4 int32, 6 pointers, double, 3 pointers, double, 4 int32, pointer
    assert ctypes.sizeof(oci.Problem) == 16 + 6 * 8 + 8 + 3 * 8 + 8 + 16 + 8
    assert oci.Stats.t.offset == 8 + 8 + 8 + 16


BAD = [
    dict(dt=0.0), dict(dt=float("nan")), dict(tol=-1.0), dict(max_iter=0), dict(N=3), dict(N=0), dict(G=0),
    dict(J=0), dict(n_mat=0),
]


@pytest.mark.parametrize("kw", BAD)
def test_invalid_problems_rejected(lib, kw):
    p = W.random_slab(1, 8, 4, 1)
    fields = dict(J=p.J, N=p.N, G=p.G, n_mat=p.n_mat, dt=p.dt, tol=p.tol, max_iter=p.max_iter)
    fields.update(kw)
    keep = [p.dx, p.mat, p.sigma_t, p.sigma_s, p.v]
    cp = oci.Problem(fields["J"], fields["N"], fields["G"], fields["n_mat"], keep[0].ctypes.data, keep[1].ctypes.data,
                     keep[2].ctypes.data, keep[3].ctypes.data, keep[4].ctypes.data, None, fields["dt"], None, None,
                     None, fields["tol"], fields["max_iter"], 0, 0, 0, None)
    h = ctypes.c_void_p()
    assert lib.oci_setup(ctypes.byref(cp), ctypes.byref(h)) == oci.E_INVAL
    assert not h.value
    assert lib.oci_last_error()


@pytest.mark.parametrize("field,val", [("dx", -0.1), ("sigma_t", -1.0), ("sigma_s", float("inf")), ("v", 0.0),
                                       ("mat", 7)])
def test_invalid_arrays_rejected(lib, field, val):
    p = W.random_slab(2, 8, 4, 2)
    arr = getattr(p, field).copy()
    arr.flat[0] = val
    with pytest.raises(oci.OCIError) as ei:
        oci.Solver(p.replace(**{field: arr}))
    assert ei.value.code == oci.E_INVAL


def test_null_handle_rejected(lib):
    st = oci.Stats()
    assert lib.oci_step(None, ctypes.byref(st)) == oci.E_INVAL
    lib.oci_destroy(None)


def test_batch_setup_validates_before_device_work(lib):
    p = W.random_slab(3, 8, 4, 1)
    keep = []
    arr = (oci.Problem * 2)(oci._problem_struct(p, keep, oci.FP64, 0, None),
                            oci._problem_struct(p, keep, oci.FP32_IR, 0, None))
    h = ctypes.c_void_p()
    assert lib.oci_batch_setup(arr, 2, ctypes.byref(h)) == oci.E_INVAL
    assert b"one precision" in lib.oci_last_error()
    assert lib.oci_batch_setup(arr, 0, ctypes.byref(h)) == oci.E_INVAL
    tc = (oci.Problem * 1)(oci._problem_struct(p, keep, oci.TF32_IR, 0, None))
    assert lib.oci_batch_setup(tc, 1, ctypes.byref(h)) == oci.E_INVAL


def test_fourier_tool_validates_before_device_work(lib):
    d = np.array([0.1]); t = np.array([0.1]); c = np.array([0.9]); out = np.zeros(1)
    args = lambda **k: (k.get("kind", 0), k.get("N", 8), k.get("n", 1), oci._ptr(d), oci._ptr(t), oci._ptr(c),
                        k.get("nt", 10), oci._ptr(out, writable=True), None)
    assert lib.oci_fourier_rho(*args(kind=3)) == oci.E_INVAL
    assert lib.oci_fourier_rho(*args(kind=-1)) == oci.E_INVAL
    assert lib.oci_fourier_rho(*args(N=3)) == oci.E_INVAL
    assert lib.oci_fourier_rho(*args(N=34)) == oci.E_INVAL
    assert lib.oci_fourier_rho(*args(n=0)) == oci.E_INVAL
    assert lib.oci_fourier_rho(*args(nt=0)) == oci.E_INVAL
    bad = np.array([-1.0])
    assert lib.oci_fourier_rho(0, 8, 1, oci._ptr(bad), oci._ptr(t), oci._ptr(c), 10, oci._ptr(out, writable=True),
                               None) == oci.E_INVAL
