"""CPU FP64 oracle for OCI and SI on the SCB x MB slab discretisation.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and
by the CPU-baseline leg of the benchmark; the product library never imports,
links or calls it, and it shares no code with the CUDA path.

Contents
  oci_oracle.c  plain C: Gauss-Legendre quadrature, dense A_j (Eqs. Aja, Aj,
                scatter, fullOCIlhs), LU with partial pivoting, OCI sweep
                (Eq. oci, Algorithm 2), red-black OCI sweep (block Gauss-Seidel
                in red-black cell order, Sec. 1), SI sweep (Algorithm 1, App. A),
                stop rule (Sec. 2.1), balance tallies (sums of Eqs. scb-mb-a..d).
  brute.py      global direct solve assembled straight from Eqs. scb-mb-a..d
                and the two closures (no iteration, no lagging).
  fourier.py    Fourier iteration matrices T_OCI, T_SI (Sec. 2.3) and the
                time-march matrix K (Sec. 2.2).
Pins for each function are in tests/test_oracle_*.py; parity unpinned: none.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oci_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboci_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INVAL, NOMEM, NOCONV, SINGULAR = 0, -1, -2, -4, -5
OCI, SI, RB = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, FP contraction off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Prob(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("N", ctypes.c_int32), ("G", ctypes.c_int32),
                ("n_mat", ctypes.c_int32),
                ("dx", ctypes.c_void_p), ("mat", ctypes.c_void_p), ("sigma_t", ctypes.c_void_p),
                ("sigma_s", ctypes.c_void_p), ("v", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("dt", ctypes.c_double), ("inc_left", ctypes.c_void_p), ("inc_right", ctypes.c_void_p),
                ("n_slots", ctypes.c_int32), ("slot_of_cell", ctypes.c_void_p),
                ("slot_first_cell", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
            L.orc_gauss_legendre.argtypes = [i32, vp, vp]
            L.orc_cell_matrix.argtypes = [vp, vp, vp, i32, vp]
            L.orc_factor_all.argtypes = [vp, vp, vp, vp, vp]
            L.orc_lu_factor.argtypes = [i32, vp, vp]
            L.orc_lu_solve.argtypes = [i32, vp, vp, vp]
            L.orc_rhs.argtypes = [vp, vp, i32, vp, vp, vp]
            L.orc_oci_cells.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
            L.orc_step.argtypes = [vp, i32, dbl, i32, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_iterate.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp]
            L.orc_balance.argtypes = [vp, vp, vp, vp, vp, vp]
            L.orc_scalar_flux.argtypes = [vp, vp, vp, vp]
            L.orc_set_threads.argtypes = [i32]
            L.orc_get_threads.restype = i32
            _lib = L
        return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (timing only)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _p(a):
    return None if a is None else a.ctypes.data


def gauss_legendre(N: int):
    mu = np.zeros(N)
    w = np.zeros(N)
    lib().orc_gauss_legendre(N, _p(mu), _p(w))
    return mu, w


class Oracle:
    """One slab problem held by the oracle: quadrature, factored A_j for every
    cell, the carried psi_{k-1/2} and the current iterate Psi."""

    def __init__(self, prob, factor: bool = True, share_factors: bool = False):
        """share_factors: factor A_j once per distinct (material, dx) pair and
        let every cell of that pair use it (bit-identical A_j, so bit-identical
        results; needed where one factor per cell would not fit in memory)."""
        self.prob = prob
        P = prob
        self._keep = dict(dx=P.dx, mat=P.mat, st=P.sigma_t, ss=P.sigma_s, v=P.v, Q=P.Q,
                          il=P.inc_left, ir=P.inc_right, slot=None, first=None)
        self.n_slots = P.J
        if share_factors:
            key = np.stack([np.asarray(P.mat, np.int64), np.asarray(P.dx, np.float64).view(np.int64)], axis=1)
            _, first, slot = np.unique(key, axis=0, return_index=True, return_inverse=True)
            self._keep["slot"] = np.ascontiguousarray(slot.reshape(-1), np.int32)
            self._keep["first"] = np.ascontiguousarray(first, np.int32)
            self.n_slots = len(first)
        self._mk_struct()
        self.mu, self.w = gauss_legendre(P.N)
        self.n = 4 * P.N * P.G
        self.LU = None
        self.piv = None
        if factor:
            self.factor()
        self.psi_prev = (np.zeros((P.J, P.G, P.N, 2)) if P.psi_init is None
                         else np.array(P.psi_init, dtype=np.float64, copy=True))
        self.Psi = np.zeros((P.J, P.G, P.N, 4))
        self.t = 0.0

    def _mk_struct(self):
        k = self._keep
        self.cp = _Prob(self.prob.J, self.prob.N, self.prob.G, self.prob.n_mat, _p(k["dx"]), _p(k["mat"]),
                        _p(k["st"]), _p(k["ss"]), _p(k["v"]), _p(k["Q"]), float(self.prob.dt),
                        _p(k["il"]), _p(k["ir"]), int(self.n_slots), _p(k["slot"]), _p(k["first"]))

    def set_boundary(self, inc_left, inc_right):
        P = self.prob
        self._keep["il"] = None if inc_left is None else np.ascontiguousarray(inc_left, np.float64).reshape(P.G, P.N, 2)
        self._keep["ir"] = None if inc_right is None else np.ascontiguousarray(inc_right, np.float64).reshape(P.G, P.N, 2)
        self._mk_struct()

    def factor(self):
        P = self.prob
        self.LU = np.zeros((self.n_slots, self.n, self.n))
        self.piv = np.zeros((self.n_slots, self.n), np.int32)
        rc = lib().orc_factor_all(ctypes.byref(self.cp), _p(self.mu), _p(self.w), _p(self.LU), _p(self.piv))
        if rc != OK:
            raise RuntimeError(f"oracle factorisation failed ({rc})")

    def cell_matrix(self, j: int) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        lib().orc_cell_matrix(ctypes.byref(self.cp), _p(self.mu), _p(self.w), int(j), _p(A))
        return A

    def rhs(self, j: int, Psi_l=None) -> np.ndarray:
        b = np.zeros(self.n)
        Psi_l = self.Psi if Psi_l is None else np.ascontiguousarray(Psi_l, np.float64)
        lib().orc_rhs(ctypes.byref(self.cp), _p(self.mu), int(j), _p(self.psi_prev), _p(Psi_l), _p(b))
        return b

    def step(self, method: int = OCI, tol=None, max_iter=None, guess=None):
        """One time step; returns dict(status, iters, e, rho, phi, bal, e_hist)."""
        P = self.prob
        tol = P.tol if tol is None else tol
        max_iter = P.max_iter if max_iter is None else max_iter
        guess = P.guess if guess is None else guess
        if guess == 1:
            self.Psi[...] = 0.0
        phi = np.zeros((P.J, P.G, 4))
        bal = np.zeros((P.G, 2, 5))
        stats = np.zeros(3)
        eh = np.zeros(max_iter)
        rc = lib().orc_step(ctypes.byref(self.cp), method, float(tol), int(max_iter),
                            _p(self.LU) if method != SI else None, _p(self.piv) if method != SI else None,
                            _p(self.psi_prev), _p(self.Psi), _p(phi), _p(bal), _p(stats), _p(eh))
        it = int(stats[0])
        if rc == OK:
            self.t += P.dt
        return dict(status=rc, iters=it, e=stats[1], rho=stats[2], phi=phi, bal=bal, e_hist=eh[:it],
                    Psi=self.Psi.copy())

    def iterate(self, n: int, method: int = OCI):
        eh = np.zeros(max(n, 1))
        rc = lib().orc_iterate(ctypes.byref(self.cp), method, int(n),
                               _p(self.LU) if method != SI else None, _p(self.piv) if method != SI else None,
                               _p(self.psi_prev), _p(self.Psi), _p(eh))
        if rc != OK:
            raise RuntimeError(f"oracle iterate failed ({rc})")
        return eh[:n]

    def cells(self, cells, Psi_l=None) -> np.ndarray:
        """A_j^{-1} b_j(Psi_l) for the listed cells only (factors them on the fly)."""
        P = self.prob
        cells = np.ascontiguousarray(cells, np.int32)
        Psi_l = self.Psi if Psi_l is None else np.ascontiguousarray(Psi_l, np.float64)
        out = np.zeros((len(cells), P.G, P.N, 4))
        rc = lib().orc_oci_cells(ctypes.byref(self.cp), _p(self.mu), _p(self.w), _p(self.psi_prev), _p(Psi_l),
                                 len(cells), _p(cells), _p(out))
        if rc != OK:
            raise RuntimeError(f"oracle cells failed ({rc})")
        return out

    def phi(self, Psi=None) -> np.ndarray:
        P = self.prob
        Psi = self.Psi if Psi is None else np.ascontiguousarray(Psi, np.float64)
        out = np.zeros((P.J, P.G, 4))
        lib().orc_scalar_flux(ctypes.byref(self.cp), _p(self.w), _p(Psi), _p(out))
        return out

    def balance(self, psi_prev, Psi) -> np.ndarray:
        P = self.prob
        out = np.zeros((P.G, 2, 5))
        lib().orc_balance(ctypes.byref(self.cp), _p(self.mu), _p(self.w),
                          _p(np.ascontiguousarray(psi_prev, np.float64)), _p(np.ascontiguousarray(Psi, np.float64)),
                          _p(out))
        return out


def balance_residual(bal: np.ndarray) -> np.ndarray:
    """[G][2] residual time + leak + collision - scatter_in - source, and the
    same divided by the sum of the terms' magnitudes."""
    r = bal[..., 0] + bal[..., 1] + bal[..., 2] - bal[..., 3] - bal[..., 4]
    scale = np.abs(bal).sum(axis=-1)
    rel = np.where(scale > 0, np.abs(r) / np.where(scale > 0, scale, 1.0), 0.0)
    return r, rel
