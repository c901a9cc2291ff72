"""ctypes binding of liboci (include/oci.h) -- argument marshalling only.

Every step of the OCI/SI path runs in liboci's CUDA kernels; this module only
converts numpy arrays / torch tensors into pointers and status codes into
exceptions.  It never falls back to another implementation: if liboci.so is not
built, `load()` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import workloads as _W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liboci.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_NOCONV, E_SINGULAR, E_NONFINITE, E_TIMEOUT, E_STATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, TF32_IR, BF16X3_IR, FP32_IR = 0, 1, 2, 3
GUESS_PREV, GUESS_ZERO, GUESS_USER = 0, 1, 2
SOLVER_AUTO, SOLVER_STRUCTURED, SOLVER_DENSE_LU = 0, 1, 2
ORDER_JACOBI, ORDER_RED_BLACK = 0, 1
SI_SEQUENTIAL, SI_SCAN = 0, 1

EXPORTS = ["oci_setup", "oci_step", "oci_solve_transient", "si_sweep", "oci_iterate", "oci_iterate_part", "si_iterate",
           "oci_get_psi", "oci_set_psi", "oci_get_phi", "oci_get_state", "oci_set_state", "oci_get_balance",
           "oci_set_boundary", "oci_set_ordering", "oci_set_si_mode", "oci_get_e_hist", "oci_get_edges", "oci_commit", "oci_get_info", "oci_destroy", "oci_last_error",
           "oci_probe_fp64_peak", "oci_batch_setup", "oci_batch_step", "oci_batch_size", "oci_batch_get_psi",
           "oci_batch_get_phi", "oci_batch_get_balance", "oci_diff_norm_noalloc", "oci_fourier_rho",
           "oci_set_acceleration"]


class OCIError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liboci error {code}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("N", ctypes.c_int32), ("G", ctypes.c_int32), ("n_mat", ctypes.c_int32),
                ("dx", ctypes.c_void_p), ("mat", ctypes.c_void_p), ("sigma_t", ctypes.c_void_p),
                ("sigma_s", ctypes.c_void_p), ("v", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("dt", ctypes.c_double), ("psi_init", ctypes.c_void_p), ("inc_left", ctypes.c_void_p),
                ("inc_right", ctypes.c_void_p), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("guess", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int32), ("cells_per_block", ctypes.c_int32), ("angle_chunks", ctypes.c_int32),
                ("inner_kernel", ctypes.c_int32), ("tuned_sweep_us", ctypes.c_double),
                ("sweep_kernel", ctypes.c_int32), ("multi_sweep", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("e_last", ctypes.c_double),
                ("rho_e_last", ctypes.c_double), ("balance_rel", ctypes.c_double * 2), ("t", ctypes.c_double),
                ("seconds", ctypes.c_double), ("refinements", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return dict(iters=self.iters, status=self.status, e=self.e_last, rho=self.rho_e_last,
                    balance_rel=(self.balance_rel[0], self.balance_rel[1]), t=self.t, seconds=self.seconds,
                    refinements=self.refinements)


_lib = None


def load(path: Optional[str] = None):
    """Load liboci.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"liboci.so not found at {p}; build it with paper_2503_00264_gb300.build.build()")
    L = ctypes.CDLL(p)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    L.oci_setup.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(vp)]
    L.oci_step.argtypes = [vp, ctypes.POINTER(Stats)]
    L.oci_solve_transient.argtypes = [vp, i32, vp, ctypes.POINTER(Stats)]
    L.si_sweep.argtypes = [vp, ctypes.POINTER(Stats)]
    L.oci_iterate.argtypes = [vp, i32, vp]
    L.oci_iterate_part.argtypes = [vp, i32, vp]
    L.si_iterate.argtypes = [vp, i32, vp]
    for f in ("oci_get_psi", "oci_set_psi", "oci_get_phi", "oci_get_balance"):
        getattr(L, f).argtypes = [vp, vp]
    L.oci_get_state.argtypes = [vp, vp, ctypes.POINTER(dbl)]
    L.oci_set_state.argtypes = [vp, vp, dbl]
    L.oci_set_boundary.argtypes = [vp, vp, vp]
    L.oci_get_e_hist.argtypes = [vp, vp, ctypes.POINTER(i32)]
    L.oci_get_edges.argtypes = [vp, vp, vp]
    L.oci_set_ordering.argtypes = [vp, i32]
    L.oci_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.oci_set_si_mode.argtypes = [vp, i32]
    L.oci_commit.argtypes = [vp, ctypes.POINTER(Stats)]
    L.oci_destroy.argtypes = [vp]
    L.oci_destroy.restype = None
    L.oci_last_error.restype = ctypes.c_char_p
    L.oci_probe_fp64_peak.argtypes = [ctypes.POINTER(dbl)]
    L.oci_batch_setup.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(vp)]
    L.oci_batch_step.argtypes = [vp, ctypes.POINTER(Stats)]
    L.oci_batch_size.argtypes = [vp, ctypes.POINTER(i32)]
    for f in ("oci_batch_get_psi", "oci_batch_get_phi", "oci_batch_get_balance"):
        getattr(L, f).argtypes = [vp, i32, vp]
    L.oci_fourier_rho.argtypes = [i32, i32, i32, vp, vp, vp, i32, vp, vp]
    L.oci_set_acceleration.argtypes = [vp, i32, i32, dbl]
    for f in EXPORTS:
        if f not in ("oci_destroy", "oci_last_error"):
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, allow=()):
    if rc != OK and rc not in allow:
        raise OCIError(rc, _lib.oci_last_error().decode())
    return rc


def _ptr(x, dtype=np.float64, writable=False):
    """Pointer of a contiguous numpy array or torch tensor (host or CUDA)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous and x.dtype == dtype):
        raise ValueError(f"expected a C-contiguous {np.dtype(dtype)} array")
    if writable and not x.flags.writeable:
        raise ValueError("array is read-only")
    return x.ctypes.data


FOURIER_OCI, FOURIER_SI, FOURIER_MARCH = 0, 1, 2
ACCEL_NONE, ACCEL_GMRES = 0, 1


def fourier_rho(kind: int, N: int, delta, tau, c, n_theta: int = 250, stream=None) -> np.ndarray:
    """Fourier spectral radius of the OCI or SI iteration, or the largest
    time-march amplification (oci_fourier_rho), for the model problems
    (delta[i], tau[i], c[i]): max over n_theta wave numbers."""
    L = load()
    d = np.ascontiguousarray(np.atleast_1d(delta), np.float64)
    t = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(tau), d.shape), np.float64)
    cc = None if c is None else np.ascontiguousarray(np.broadcast_to(np.atleast_1d(c), d.shape), np.float64)
    out = np.zeros(d.shape)
    _check(L.oci_fourier_rho(int(kind), int(N), int(d.size), _ptr(d), _ptr(t), _ptr(cc), int(n_theta),
                             _ptr(out, writable=True), stream))
    return out


def current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # torch absent or no GPU: use the legacy default stream
        pass
    return None


def fp64_peak() -> float:
    L = load()
    v = ctypes.c_double(0.0)
    _check(L.oci_probe_fp64_peak(ctypes.byref(v)))
    return v.value


def _problem_struct(P, keep, precision, solver, stream, tol=None, max_iter=None, guess=None):
    k = [np.ascontiguousarray(a) if a is not None else None
         for a in (P.dx, P.mat, P.sigma_t, P.sigma_s, P.v, P.Q, P.psi_init, P.inc_left, P.inc_right)]
    keep.append(k)
    return Problem(P.J, P.N, P.G, P.n_mat, _ptr(k[0]), _ptr(k[1], np.int32), _ptr(k[2]), _ptr(k[3]),
                   _ptr(k[4]), _ptr(k[5]), float(P.dt), _ptr(k[6]), _ptr(k[7]), _ptr(k[8]),
                   float(P.tol if tol is None else tol), int(P.max_iter if max_iter is None else max_iter),
                   int(precision), int(P.guess if guess is None else guess), int(solver), stream)


class BatchSolver:
    """Many independent slabs advanced together (oci_batch_* calls); precision
    FP64 or FP32_IR (one for the whole batch)."""

    def __init__(self, probs, stream=None, precision: int = FP64):
        self.L = load()
        self.probs = list(probs)
        self._keep = []
        st = current_stream() if stream is None else stream
        arr = (Problem * len(self.probs))(
            *[_problem_struct(p, self._keep, precision, SOLVER_AUTO, st) for p in self.probs])
        self._arr = arr
        h = ctypes.c_void_p()
        _check(self.L.oci_batch_setup(arr, len(self.probs), ctypes.byref(h)))
        self.h = h

    def step(self, allow_noconv: bool = False):
        st = (Stats * len(self.probs))()
        _check(self.L.oci_batch_step(self.h, st), (E_NOCONV,) if allow_noconv else ())
        return [st[i].as_dict() for i in range(len(self.probs))]

    def psi(self, s: int):
        P = self.probs[s]
        out = np.zeros((P.J, P.G, P.N, 4))
        _check(self.L.oci_batch_get_psi(self.h, int(s), _ptr(out, writable=True)))
        return out

    def phi(self, s: int):
        P = self.probs[s]
        out = np.zeros((P.J, P.G, 4))
        _check(self.L.oci_batch_get_phi(self.h, int(s), _ptr(out, writable=True)))
        return out

    def balance(self, s: int):
        P = self.probs[s]
        out = np.zeros((P.G, 2, 5))
        _check(self.L.oci_batch_get_balance(self.h, int(s), _ptr(out, writable=True)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.L.oci_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One slab problem on the GPU (an oci_handle)."""

    def __init__(self, prob: "_W.Problem", precision: int = FP64, solver: int = SOLVER_AUTO, stream=None,
                 tol: Optional[float] = None, max_iter: Optional[int] = None, guess: Optional[int] = None):
        self.L = load()
        P = prob
        self.prob = P
        self._keep = [np.ascontiguousarray(a) if a is not None else None
                      for a in (P.dx, P.mat, P.sigma_t, P.sigma_s, P.v, P.Q, P.psi_init, P.inc_left, P.inc_right)]
        k = self._keep
        self.cp = Problem(P.J, P.N, P.G, P.n_mat, _ptr(k[0]), _ptr(k[1], np.int32), _ptr(k[2]), _ptr(k[3]),
                          _ptr(k[4]), _ptr(k[5]), float(P.dt), _ptr(k[6]), _ptr(k[7]), _ptr(k[8]),
                          float(P.tol if tol is None else tol), int(P.max_iter if max_iter is None else max_iter),
                          int(precision), int(P.guess if guess is None else guess), int(solver),
                          current_stream() if stream is None else stream)
        h = ctypes.c_void_p()
        _check(self.L.oci_setup(ctypes.byref(self.cp), ctypes.byref(h)))
        self.h = h
        self.J, self.N, self.G = P.J, P.N, P.G

    # --------------------------------------------------------------- stepping
    def step(self, allow_noconv: bool = False) -> dict:
        st = Stats()
        rc = self.L.oci_step(self.h, ctypes.byref(st))
        _check(rc, (E_NOCONV,) if allow_noconv else ())
        return st.as_dict()

    def si_step(self, allow_noconv: bool = False) -> dict:
        st = Stats()
        rc = self.L.si_sweep(self.h, ctypes.byref(st))
        _check(rc, (E_NOCONV,) if allow_noconv else ())
        return st.as_dict()

    def solve_transient(self, n_steps: int, phi_out=None):
        st = (Stats * max(n_steps, 1))()
        _check(self.L.oci_solve_transient(self.h, int(n_steps), _ptr(phi_out, writable=True), st))
        return [st[k].as_dict() for k in range(n_steps)]

    def iterate(self, n: int, e_hist=None) -> np.ndarray:
        out = np.zeros(max(n, 1)) if e_hist is None else e_hist
        _check(self.L.oci_iterate(self.h, int(n), _ptr(out, writable=True)))
        return out[:n] if e_hist is None else out

    def iterate_part(self, part: int, e_out=None):
        """One sweep in two calls (oci_iterate_part): part 0 sweeps the interior
        blocks and returns at once; part 1 sweeps the two end blocks and writes e
        of the whole sweep into e_out (numpy or a torch tensor of one double, host
        or device), if given."""
        _check(self.L.oci_iterate_part(self.h, int(part), _ptr(e_out, writable=True) if e_out is not None else None))

    def si_iterate(self, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1))
        _check(self.L.si_iterate(self.h, int(n), _ptr(out, writable=True)))
        return out[:n]

    # --------------------------------------------------------------- state
    def psi(self, out=None):
        out = np.zeros((self.J, self.G, self.N, 4)) if out is None else out
        _check(self.L.oci_get_psi(self.h, _ptr(out, writable=True)))
        return out

    def set_psi(self, psi):
        _check(self.L.oci_set_psi(self.h, _ptr(np.ascontiguousarray(psi, np.float64) if isinstance(psi, np.ndarray) else psi)))

    def phi(self, out=None):
        out = np.zeros((self.J, self.G, 4)) if out is None else out
        _check(self.L.oci_get_phi(self.h, _ptr(out, writable=True)))
        return out

    def state(self):
        pp = np.zeros((self.J, self.G, self.N, 2))
        t = ctypes.c_double()
        _check(self.L.oci_get_state(self.h, _ptr(pp, writable=True), ctypes.byref(t)))
        return pp, t.value

    def state_into(self, out) -> float:
        """psi_prev into a caller buffer ([J][G][N][2], host or device); returns t."""
        t = ctypes.c_double()
        _check(self.L.oci_get_state(self.h, _ptr(out, writable=True), ctypes.byref(t)))
        return t.value

    def set_state(self, psi_prev, t: float):
        arr = None if psi_prev is None else (np.ascontiguousarray(psi_prev, np.float64)
                                             if isinstance(psi_prev, np.ndarray) else psi_prev)
        _check(self.L.oci_set_state(self.h, _ptr(arr), float(t)))

    def balance(self) -> np.ndarray:
        out = np.zeros((self.G, 2, 5))
        _check(self.L.oci_get_balance(self.h, _ptr(out, writable=True)))
        return out

    def set_boundary(self, inc_left, inc_right):
        """Incident fluxes [G][N][2] (numpy, or torch tensors on the host or the device)."""
        def arr(x):
            if x is None or hasattr(x, "data_ptr"):
                return x
            return np.ascontiguousarray(x, np.float64)
        _check(self.L.oci_set_boundary(self.h, _ptr(arr(inc_left)), _ptr(arr(inc_right))))

    def e_hist(self) -> np.ndarray:
        n = ctypes.c_int32()
        _check(self.L.oci_get_e_hist(self.h, None, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1))
        _check(self.L.oci_get_e_hist(self.h, _ptr(out, writable=True), ctypes.byref(n)))
        return out[: n.value]

    def info(self) -> dict:
        i = Info()
        _check(self.L.oci_get_info(self.h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def set_si_mode(self, mode: int):
        _check(self.L.oci_set_si_mode(self.h, int(mode)))

    def set_acceleration(self, accel: int, restart: int = 20, residual_factor: float = 0.05):
        _check(self.L.oci_set_acceleration(self.h, int(accel), int(restart), float(residual_factor)))

    def set_ordering(self, ordering: int):
        _check(self.L.oci_set_ordering(self.h, int(ordering)))

    def edges(self, left=None, right=None):
        """Edge values [G][N][2] of cell 0 (kL, hL) and cell J-1 (kR, hR), into the
        given buffers (numpy, or torch tensors on the host or the device) or new arrays."""
        left = np.zeros((self.G, self.N, 2)) if left is None else left
        right = np.zeros((self.G, self.N, 2)) if right is None else right
        _check(self.L.oci_get_edges(self.h, _ptr(left, writable=True), _ptr(right, writable=True)))
        return left, right

    def commit(self) -> dict:
        st = Stats()
        _check(self.L.oci_commit(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.L.oci_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
