"""Python access to the plain FP64 CPU oracle (``mnl_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module.  The library's product path never
imports it.

Every function takes a ``datagen.Problem``-like object (attributes N, K, p, d,
f, gamma_base, X, Y, Z, choice and, optionally, w: float32 observation weights)
and float64 coefficient vectors in the order of eq. "theta vec".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mnl_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_mnl.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, OpenMP); returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int32), ("p", C.c_int32), ("d", C.c_int32), ("f", C.c_int32),
                ("gamma_base", C.c_int32), ("X", C.c_void_p), ("Y", C.c_void_p), ("Z", C.c_void_p),
                ("choice", C.c_void_p), ("w", C.c_void_p)]


class FitOpts(C.Structure):
    _fields_ = [("maxiter", C.c_int32), ("max_halvings", C.c_int32), ("gtol", C.c_double), ("ftol", C.c_double),
                ("steptol", C.c_double), ("nthreads", C.c_int32), ("ls_rel_tol", C.c_double)]


class FitStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("ls_evals", C.c_int32), ("stop", C.c_int32), ("pad", C.c_int32),
                ("loglik", C.c_double), ("grad_inf", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            dp = C.POINTER(C.c_double)
            lib.oracle_num_params.restype = C.c_int64
            lib.oracle_num_params.argtypes = [C.c_int] * 5
            lib.oracle_probs.argtypes = [P, dp, dp, dp]
            lib.oracle_loglik_grad.argtypes = [P, dp, dp, dp]
            lib.oracle_neg_hessian.argtypes = [P, dp, dp, C.c_int]
            lib.oracle_neg_hessian_entries.argtypes = [P, dp, C.c_int64, C.POINTER(C.c_int64),
                                                       C.POINTER(C.c_int64), dp, C.c_int]
            lib.oracle_cholesky.argtypes = [C.c_int64, dp]
            lib.oracle_cholesky_solve.argtypes = [C.c_int64, dp, dp]
            lib.oracle_fit.argtypes = [P, C.POINTER(FitOpts), dp, C.POINTER(FitStats)]
            lib.oracle_check.argtypes = [P]
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Keep:
    """Holds the C struct plus the arrays it points into."""

    def __init__(self, prob):
        self.X = np.ascontiguousarray(prob.X, dtype=np.float32)
        self.Y = np.ascontiguousarray(prob.Y, dtype=np.float32)
        self.Z = np.ascontiguousarray(prob.Z, dtype=np.float32)
        self.c = np.ascontiguousarray(prob.choice, dtype=np.int32)
        w = getattr(prob, "w", None)
        self.w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        self.s = _Problem(prob.N, prob.K, prob.p, prob.d, prob.f, prob.gamma_base, self.X.ctypes.data,
                          self.Y.ctypes.data, self.Z.ctypes.data, self.c.ctypes.data,
                          None if self.w is None else self.w.ctypes.data)
        self.n = num_params(prob.K, prob.p, prob.d, prob.f, prob.gamma_base)


def num_params(K, p, d, f, gamma_base=0) -> int:
    return int(_load().oracle_num_params(K, p, d, f, gamma_base))


def _theta(prob, theta, n):
    if theta is None:
        return np.zeros(n)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    if t.shape != (n,):
        raise ValueError(f"theta must have shape ({n},)")
    return t


def check(prob) -> int:
    k = _Keep(prob)
    return int(_load().oracle_check(C.byref(k.s)))


def probs(prob, theta=None):
    """P [N][K] and l."""
    k = _Keep(prob)
    t = _theta(prob, theta, k.n)
    P = np.empty((prob.N, prob.K))
    l = C.c_double()
    rc = _load().oracle_probs(C.byref(k.s), _dptr(t), _dptr(P), C.byref(l))
    if rc:
        raise ValueError(f"oracle_probs failed ({rc})")
    return P, l.value


def loglik_grad(prob, theta=None):
    """(l, g)."""
    k = _Keep(prob)
    t = _theta(prob, theta, k.n)
    g = np.empty(k.n)
    l = C.c_double()
    rc = _load().oracle_loglik_grad(C.byref(k.s), _dptr(t), C.byref(l), _dptr(g))
    if rc:
        raise ValueError(f"oracle_loglik_grad failed ({rc})")
    return l.value, g


def loglik(prob, theta=None) -> float:
    k = _Keep(prob)
    t = _theta(prob, theta, k.n)
    l = C.c_double()
    rc = _load().oracle_loglik_grad(C.byref(k.s), _dptr(t), C.byref(l), None)
    if rc:
        raise ValueError(f"oracle_loglik_grad failed ({rc})")
    return l.value


def neg_hessian(prob, theta=None, nthreads: int = 0) -> np.ndarray:
    """F = -H, full symmetric [n][n]."""
    k = _Keep(prob)
    t = _theta(prob, theta, k.n)
    F = np.empty((k.n, k.n))
    rc = _load().oracle_neg_hessian(C.byref(k.s), _dptr(t), _dptr(F), nthreads)
    if rc:
        raise ValueError(f"oracle_neg_hessian failed ({rc})")
    return F


def neg_hessian_entries(prob, theta, rows, cols, nthreads: int = 0) -> np.ndarray:
    """Selected entries of F = -H, each summed over all observations."""
    k = _Keep(prob)
    t = _theta(prob, theta, k.n)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    if r.shape != c.shape or r.ndim != 1 or (r.size and (min(r.min(), c.min()) < 0 or max(r.max(), c.max()) >= k.n)):
        raise ValueError("bad entry lists")
    out = np.empty(r.size)
    rc = _load().oracle_neg_hessian_entries(C.byref(k.s), _dptr(t), r.size, r.ctypes.data_as(C.POINTER(C.c_int64)),
                                            c.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(out), nthreads)
    if rc:
        raise ValueError(f"oracle_neg_hessian_entries failed ({rc})")
    return out


def cholesky(A: np.ndarray):
    """Lower Cholesky factor of a symmetric positive definite matrix, or None if not PD."""
    L = np.array(A, dtype=np.float64, order="C", copy=True)
    n = L.shape[0]
    rc = _load().oracle_cholesky(n, _dptr(L))
    return None if rc else L


def cholesky_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.array(b, dtype=np.float64, copy=True)
    _load().oracle_cholesky_solve(L.shape[0], _dptr(L), _dptr(x))
    return x


STOP_NAMES = {1: "gtol", 2: "ftol", 3: "steptol", 4: "maxiter", -2: "not_pd", -4: "linesearch"}


def std_errors(prob, theta) -> np.ndarray:
    """Asymptotic standard errors at theta (normally the estimate): the square roots of the diagonal of the
    inverse of the observed information F = -H (the coefficient table of the package's ``summary`` method,
    Sec. 2.3).  Each diagonal entry of F^-1 comes from one solve with the oracle's Cholesky factor."""
    F = neg_hessian(prob, theta)
    L = cholesky(F)
    if L is None:
        raise ValueError("-H is not positive definite at theta")
    n = F.shape[0]
    var = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        var[i] = cholesky_solve(L, e)[i]
    return np.sqrt(var)

# Rounding-noise allowance of the line search: 8 units of FP64 roundoff times |l|.
LS_REL_TOL = 8 * 2.0 ** -53


def fit(prob, theta0=None, *, maxiter=100, max_halvings=30, gtol=1e-8, ftol=0.0, steptol=1e-12, nthreads=0,
        ls_rel_tol=LS_REL_TOL):
    """Newton-Raphson with step halving.  Returns (theta_hat, stats dict)."""
    k = _Keep(prob)
    t = np.array(_theta(prob, theta0, k.n), copy=True)
    o = FitOpts(maxiter, max_halvings, gtol, ftol, steptol, nthreads, ls_rel_tol)
    st = FitStats()
    rc = _load().oracle_fit(C.byref(k.s), C.byref(o), _dptr(t), C.byref(st))
    stats = dict(rc=rc, iters=st.iters, ls_evals=st.ls_evals, stop=STOP_NAMES.get(st.stop, st.stop),
                 loglik=st.loglik, grad_inf=st.grad_inf)
    if rc not in (0,):
        raise RuntimeError(f"oracle_fit failed: {stats}")
    return t, stats
