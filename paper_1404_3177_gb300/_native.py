"""ctypes binding of ``include/mnl.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own.  Loading fails loudly when the CUDA library has not been
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

MNL_OK = 0
MNL_ERR_INVALID_ARG = 1
MNL_ERR_OOM = 2
MNL_ERR_CUDA = 3
MNL_ERR_NOT_PD = 4
MNL_ERR_NONFINITE = 5
MNL_ERR_LINESEARCH = 6
MNL_MAXITER = 7
MNL_ERR_TIMEOUT = 8
MNL_ERR_UNSUPPORTED = 9
MNL_PENDING = 10

MNL_FP64, MNL_TF32, MNL_BF16 = 0, 1, 2
PRECISIONS = {"fp64": MNL_FP64, "tf32": MNL_TF32, "bf16": MNL_BF16}

MNL_STOP_GTOL, MNL_STOP_FTOL, MNL_STOP_STEPTOL, MNL_STOP_MAXITER, MNL_STOP_NOISE = 1, 2, 3, 4, 5

# Every entry point declared in include/mnl.h.
EXPORTS = (
    "mnl_num_params", "mnl_status_string", "mnl_workspace_bytes", "mnl_fit_opts_default", "mnl_create",
    "mnl_upload", "mnl_loglik_grad", "mnl_hessian", "mnl_newton_step", "mnl_fit", "mnl_destroy",
    "mnl_loglik_grad_noalloc", "mnl_set_solve", "mnl_set_wait_bound", "mnl_set_weights",
    "mnl_create_ex", "mnl_hessian_vec", "mnl_set_cg_max", "mnl_shard_sums_size", "mnl_shard_grad_hess", "mnl_shard_solve", "mnl_shard_loglik", "mnl_loglik_roundoff", "mnl_std_errors", "mnl_predict",
    "mnl_check_collinear", "mnl_drop_columns", "mnl_batch_create", "mnl_batch_num_params", "mnl_batch_fit",
    "mnl_batch_destroy", "mnl_server_opts_default", "mnl_server_create", "mnl_server_submit", "mnl_server_step",
    "mnl_server_poll", "mnl_server_finished", "mnl_server_memory_in_use", "mnl_server_destroy",
)

MNL_SOLVE_AUTO, MNL_SOLVE_FP64, MNL_SOLVE_MIXED = 0, 1, 2
MNL_FACTOR_NONE, MNL_FACTOR_COOP, MNL_FACTOR_TENSOR = 0, 1, 2
MNL_WAIT_SYRK, MNL_WAIT_PASS, MNL_WAIT_COOP, MNL_WAIT_PANEL = 15, 16, 32, 64
SOLVES = {"auto": MNL_SOLVE_AUTO, "fp64": MNL_SOLVE_FP64, "mixed": MNL_SOLVE_MIXED}


class mnl_dims(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int32), ("p", C.c_int32), ("d", C.c_int32), ("f", C.c_int32),
                ("gamma_base", C.c_int32)]


class mnl_data(C.Structure):
    _fields_ = [("X", C.c_void_p), ("Y", C.c_void_p), ("Z", C.c_void_p), ("choice", C.c_void_p)]


class mnl_step_info(C.Structure):
    _fields_ = [("loglik_old", C.c_double), ("loglik_new", C.c_double), ("grad_inf", C.c_double),
                ("step_inf", C.c_double), ("theta_inf", C.c_double), ("step_scale", C.c_double),
                ("ls_noise", C.c_double), ("halvings", C.c_int32), ("ls_evals", C.c_int32),
                ("t_pass_ms", C.c_float), ("t_hess_ms", C.c_float), ("t_chol_ms", C.c_float),
                ("t_ls_ms", C.c_float), ("t_build_ms", C.c_float), ("t_syrk_ms", C.c_float),
                ("t_band_ms", C.c_float), ("t_zblk_ms", C.c_float), ("t_asm_ms", C.c_float),
                ("t_factor_ms", C.c_float), ("t_solve_ms", C.c_float), ("t_fallback_ms", C.c_float),
                ("launches", C.c_int32), ("solve_mode", C.c_int32), ("refine_steps", C.c_int32),
                ("fallback", C.c_int32), ("factor_kind", C.c_int32), ("wait_errors", C.c_int32),
                ("cg_iters", C.c_int32)]


class mnl_fit_opts(C.Structure):
    _fields_ = [("maxiter", C.c_int32), ("max_halvings", C.c_int32), ("gtol", C.c_double), ("ftol", C.c_double),
                ("steptol", C.c_double)]


class mnl_fit_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("ls_evals", C.c_int32), ("stop_reason", C.c_int32), ("status", C.c_int32),
                ("loglik", C.c_double), ("grad_inf", C.c_double), ("dloglik", C.c_double),
                ("step_rel", C.c_double), ("t_total_ms", C.c_double), ("t_pass_ms", C.c_double),
                ("t_hess_ms", C.c_double), ("t_chol_ms", C.c_double), ("t_ls_ms", C.c_double)]


class mnl_batch_problem_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("stop_reason", C.c_int32), ("iters", C.c_int32), ("ls_evals", C.c_int32),
                ("loglik", C.c_double), ("grad_inf", C.c_double)]


class mnl_batch_info(C.Structure):
    _fields_ = [("problems", C.POINTER(mnl_batch_problem_info)), ("iterations", C.c_int32),
                ("converged", C.c_int32), ("failed", C.c_int32), ("pass_rows", C.c_int32),
                ("t_total_ms", C.c_double), ("t_graph_ms", C.c_double)]


class mnl_server_opts(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("precision", C.c_int32), ("max_active", C.c_int32),
                ("max_skips", C.c_int32), ("pad", C.c_int32), ("fit", mnl_fit_opts)]


class mnl_request_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("stop_reason", C.c_int32), ("iters", C.c_int32), ("ls_evals", C.c_int32),
                ("loglik", C.c_double), ("grad_inf", C.c_double), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double)]


def struct_dict(s: C.Structure) -> dict:
    return {name: getattr(s, name) for name, _ in s._fields_}


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load() -> C.CDLL:
    """Load libmnl.so (built by ``_build.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"the CUDA library {path} is not built; run paper_1404_3177_gb300._build.build() "
                               "(there is no CPU fallback)")
        lib = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
        lib.mnl_num_params.restype = i64
        lib.mnl_num_params.argtypes = [C.POINTER(mnl_dims)]
        lib.mnl_status_string.restype = C.c_char_p
        lib.mnl_status_string.argtypes = [i32]
        lib.mnl_workspace_bytes.restype = C.c_size_t
        lib.mnl_workspace_bytes.argtypes = [C.POINTER(mnl_dims), i32]
        lib.mnl_fit_opts_default.restype = None
        lib.mnl_fit_opts_default.argtypes = [C.POINTER(mnl_fit_opts)]
        lib.mnl_create.restype = i32
        lib.mnl_create.argtypes = [C.POINTER(mnl_dims), C.POINTER(mnl_data), i32, vp, C.POINTER(vp)]
        lib.mnl_upload.restype = i32
        lib.mnl_upload.argtypes = [vp, C.POINTER(mnl_data)]
        lib.mnl_loglik_grad.restype = i32
        lib.mnl_loglik_grad.argtypes = [vp, vp, C.POINTER(C.c_double), vp]
        lib.mnl_hessian.restype = i32
        lib.mnl_hessian.argtypes = [vp, vp, vp]
        lib.mnl_newton_step.restype = i32
        lib.mnl_newton_step.argtypes = [vp, vp, C.POINTER(mnl_step_info)]
        lib.mnl_fit.restype = i32
        lib.mnl_fit.argtypes = [vp, C.POINTER(mnl_fit_opts), vp, C.POINTER(mnl_fit_info)]
        lib.mnl_std_errors.restype = i32
        lib.mnl_std_errors.argtypes = [vp, vp, vp]
        lib.mnl_predict.restype = i32
        lib.mnl_predict.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        lib.mnl_create_ex.restype = i32
        lib.mnl_check_collinear.argtypes = [vp, C.c_double, vp, C.POINTER(C.c_int32)]
        lib.mnl_check_collinear.restype = i32
        lib.mnl_drop_columns.argtypes = [vp, vp]
        lib.mnl_drop_columns.restype = i32
        lib.mnl_create_ex.argtypes = [C.POINTER(mnl_dims), C.POINTER(mnl_data), i32, i32, vp, C.POINTER(vp)]
        lib.mnl_hessian_vec.restype = i32
        lib.mnl_hessian_vec.argtypes = [vp, vp, vp, vp]
        lib.mnl_set_cg_max.restype = i32
        lib.mnl_set_cg_max.argtypes = [vp, C.c_int32]
        lib.mnl_shard_sums_size.restype = i64
        lib.mnl_shard_sums_size.argtypes = [C.POINTER(mnl_dims)]
        lib.mnl_shard_grad_hess.restype = i32
        lib.mnl_shard_grad_hess.argtypes = [vp, vp, vp]
        lib.mnl_shard_solve.restype = i32
        lib.mnl_shard_solve.argtypes = [vp, vp, vp, C.POINTER(mnl_step_info)]
        lib.mnl_shard_loglik.restype = i32
        lib.mnl_shard_loglik.argtypes = [vp, vp, vp, C.c_double, vp]
        lib.mnl_loglik_roundoff.restype = C.c_double
        lib.mnl_loglik_roundoff.argtypes = [vp]
        lib.mnl_set_weights.restype = i32
        lib.mnl_set_weights.argtypes = [vp, vp]
        lib.mnl_set_wait_bound.restype = i32
        lib.mnl_set_wait_bound.argtypes = [vp, C.c_uint64]
        lib.mnl_destroy.restype = i32
        lib.mnl_destroy.argtypes = [vp]
        lib.mnl_batch_create.restype = i32
        lib.mnl_batch_create.argtypes = [i32, C.POINTER(mnl_dims), C.POINTER(mnl_data), i32, vp, C.POINTER(vp)]
        lib.mnl_batch_num_params.restype = i64
        lib.mnl_batch_num_params.argtypes = [vp, C.POINTER(C.c_int64)]
        lib.mnl_batch_fit.restype = i32
        lib.mnl_batch_fit.argtypes = [vp, C.POINTER(mnl_fit_opts), vp, C.POINTER(mnl_batch_info)]
        lib.mnl_batch_destroy.restype = i32
        lib.mnl_batch_destroy.argtypes = [vp]
        lib.mnl_server_opts_default.restype = None
        lib.mnl_server_opts_default.argtypes = [C.POINTER(mnl_server_opts)]
        lib.mnl_server_create.restype = i32
        lib.mnl_server_create.argtypes = [C.POINTER(mnl_server_opts), vp, C.POINTER(vp)]
        lib.mnl_server_submit.restype = i32
        lib.mnl_server_submit.argtypes = [vp, C.POINTER(mnl_dims), C.POINTER(mnl_data), vp, C.POINTER(C.c_uint64)]
        lib.mnl_server_step.restype = i32
        lib.mnl_server_step.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        lib.mnl_server_poll.restype = i32
        lib.mnl_server_poll.argtypes = [vp, C.c_uint64, vp, C.POINTER(mnl_request_result)]
        lib.mnl_server_finished.restype = i32
        lib.mnl_server_finished.argtypes = [vp, C.POINTER(C.c_uint64), C.c_int32, C.POINTER(C.c_int32)]
        lib.mnl_server_memory_in_use.restype = C.c_size_t
        lib.mnl_server_memory_in_use.argtypes = [vp]
        lib.mnl_server_destroy.restype = i32
        lib.mnl_server_destroy.argtypes = [vp]
        lib.mnl_set_solve.restype = i32
        lib.mnl_set_solve.argtypes = [vp, i32]
        lib.mnl_loglik_grad_noalloc.restype = i32
        lib.mnl_loglik_grad_noalloc.argtypes = [C.POINTER(mnl_dims), C.POINTER(mnl_data), i32, vp, vp, vp, vp, vp,
                                                vp]
        _lib = lib
        return lib


class MnlError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {mnl_status_string(status)} (status {status})")


def _check(rc: int, where: str) -> int:
    if rc != MNL_OK and rc != MNL_MAXITER:
        raise MnlError(rc, where)
    return rc


# ---- same-name wrappers --------------------------------------------------

def mnl_status_string(status: int) -> str:
    return load().mnl_status_string(status).decode()


def mnl_num_params(dims: mnl_dims) -> int:
    return int(load().mnl_num_params(C.byref(dims)))


def mnl_workspace_bytes(dims: mnl_dims, precision: int) -> int:
    return int(load().mnl_workspace_bytes(C.byref(dims), precision))


def mnl_fit_opts_default() -> mnl_fit_opts:
    o = mnl_fit_opts()
    load().mnl_fit_opts_default(C.byref(o))
    return o


def mnl_create(dims: mnl_dims, data: mnl_data | None, precision: int, stream: int | None) -> int:
    h = C.c_void_p()
    rc = load().mnl_create(C.byref(dims), C.byref(data) if data is not None else None, precision,
                           C.c_void_p(stream or 0), C.byref(h))
    _check(rc, "mnl_create")
    return h.value


def mnl_upload(handle: int, host_data: mnl_data) -> None:
    _check(load().mnl_upload(C.c_void_p(handle), C.byref(host_data)), "mnl_upload")


def mnl_loglik_grad(handle: int, theta_ptr: int, want_loglik: bool, grad_ptr: int | None) -> float | None:
    l = C.c_double()
    rc = load().mnl_loglik_grad(C.c_void_p(handle), C.c_void_p(theta_ptr), C.byref(l) if want_loglik else None,
                                C.c_void_p(grad_ptr) if grad_ptr else None)
    _check(rc, "mnl_loglik_grad")
    return l.value if want_loglik else None


def mnl_hessian(handle: int, theta_ptr: int, H_ptr: int) -> None:
    _check(load().mnl_hessian(C.c_void_p(handle), C.c_void_p(theta_ptr), C.c_void_p(H_ptr)), "mnl_hessian")


def mnl_newton_step(handle: int, theta_ptr: int) -> mnl_step_info:
    """Raises MnlError on failure; after MNL_ERR_TIMEOUT its `info` holds the step info (wait_errors)."""
    info = mnl_step_info()
    rc = load().mnl_newton_step(C.c_void_p(handle), C.c_void_p(theta_ptr), C.byref(info))
    if rc != MNL_OK:
        err = MnlError(rc, "mnl_newton_step")
        err.info = struct_dict(info)
        raise err
    return info


def mnl_fit(handle: int, opts: mnl_fit_opts | None, theta_ptr: int) -> mnl_fit_info:
    info = mnl_fit_info()
    rc = load().mnl_fit(C.c_void_p(handle), C.byref(opts) if opts is not None else None, C.c_void_p(theta_ptr),
                        C.byref(info))
    _check(rc, "mnl_fit")
    return info


def mnl_set_solve(handle: int, mode: int) -> None:
    _check(load().mnl_set_solve(C.c_void_p(handle), mode), "mnl_set_solve")


def mnl_std_errors(handle: int, theta_ptr: int, se_ptr: int) -> None:
    _check(load().mnl_std_errors(C.c_void_p(handle), C.c_void_p(theta_ptr), C.c_void_p(se_ptr)), "mnl_std_errors")


def mnl_predict(handle: int, theta_ptr: int, P_ptr: int, want_loglik: bool = True) -> float | None:
    l = C.c_double()
    _check(load().mnl_predict(C.c_void_p(handle), C.c_void_p(theta_ptr), C.c_void_p(P_ptr),
                              C.byref(l) if want_loglik else None), "mnl_predict")
    return l.value if want_loglik else None


def mnl_check_collinear(handle: int, tol: float, nflags: int):
    """(flags, ndropped): flags is a list of nflags ints (0 kept, 1 dependent)."""
    flags = (C.c_int32 * max(nflags, 1))()
    nd = C.c_int32()
    _check(load().mnl_check_collinear(C.c_void_p(handle), C.c_double(tol), flags, C.byref(nd)),
           "mnl_check_collinear")
    return list(flags)[:nflags], nd.value


def mnl_drop_columns(handle: int, flags) -> None:
    if flags is None:
        _check(load().mnl_drop_columns(C.c_void_p(handle), None), "mnl_drop_columns")
        return
    arr = (C.c_int32 * max(len(flags), 1))(*[int(x) for x in flags])
    _check(load().mnl_drop_columns(C.c_void_p(handle), arr), "mnl_drop_columns")


MNL_CREATE_TRUNCATED = 1


def mnl_create_ex(dims: mnl_dims, data: mnl_data | None, precision: int, flags: int, stream: int | None) -> int:
    h = C.c_void_p()
    _check(load().mnl_create_ex(C.byref(dims), C.byref(data) if data is not None else None, precision, flags,
                                C.c_void_p(stream or 0), C.byref(h)), "mnl_create_ex")
    return h.value


def mnl_hessian_vec(handle: int, theta_ptr: int, v_ptr: int, Hv_ptr: int) -> None:
    _check(load().mnl_hessian_vec(C.c_void_p(handle), C.c_void_p(theta_ptr), C.c_void_p(v_ptr), C.c_void_p(Hv_ptr)),
           "mnl_hessian_vec")


def mnl_set_cg_max(handle: int, iters: int) -> None:
    _check(load().mnl_set_cg_max(C.c_void_p(handle), int(iters)), "mnl_set_cg_max")


def mnl_shard_sums_size(dims: mnl_dims) -> int:
    return int(load().mnl_shard_sums_size(C.byref(dims)))


def mnl_shard_grad_hess(handle: int, theta_ptr: int, sums_ptr: int) -> None:
    _check(load().mnl_shard_grad_hess(C.c_void_p(handle), C.c_void_p(theta_ptr), C.c_void_p(sums_ptr)),
           "mnl_shard_grad_hess")


def mnl_shard_solve(handle: int, sums_ptr: int, delta_ptr: int) -> dict:
    info = mnl_step_info()
    _check(load().mnl_shard_solve(C.c_void_p(handle), C.c_void_p(sums_ptr), C.c_void_p(delta_ptr), C.byref(info)),
           "mnl_shard_solve")
    return struct_dict(info)


def mnl_shard_loglik(handle: int, theta_ptr: int, delta_ptr: int | None, t: float, l2_ptr: int) -> None:
    _check(load().mnl_shard_loglik(C.c_void_p(handle), C.c_void_p(theta_ptr),
                                   C.c_void_p(delta_ptr) if delta_ptr else None, float(t), C.c_void_p(l2_ptr)),
           "mnl_shard_loglik")


def mnl_loglik_roundoff(handle: int) -> float:
    return float(load().mnl_loglik_roundoff(C.c_void_p(handle)))


def mnl_set_weights(handle: int, w_ptr: int | None) -> None:
    _check(load().mnl_set_weights(C.c_void_p(handle), C.c_void_p(w_ptr) if w_ptr else None), "mnl_set_weights")


def mnl_set_wait_bound(handle: int, ns: int) -> None:
    _check(load().mnl_set_wait_bound(C.c_void_p(handle), C.c_uint64(ns)), "mnl_set_wait_bound")


def mnl_destroy(handle: int) -> None:
    _check(load().mnl_destroy(C.c_void_p(handle)), "mnl_destroy")


def mnl_loglik_grad_noalloc(dims: mnl_dims, data: mnl_data, precision: int, theta_ptr: int, loglik_ptr: int,
                            grad_ptr: int, P_ptr: int, zbar_ptr: int | None, stream: int | None) -> None:
    """Enqueue l, g (and P, zbar) into caller-owned device buffers; allocates nothing."""
    rc = load().mnl_loglik_grad_noalloc(C.byref(dims), C.byref(data), precision, C.c_void_p(theta_ptr),
                                        C.c_void_p(loglik_ptr), C.c_void_p(grad_ptr), C.c_void_p(P_ptr),
                                        C.c_void_p(zbar_ptr) if zbar_ptr else None, C.c_void_p(stream or 0))
    _check(rc, "mnl_loglik_grad_noalloc")


def mnl_batch_create(dims: list, data: list, precision: int, stream: int | None) -> int:
    n = len(dims)
    da = (mnl_dims * n)(*dims)
    dd = (mnl_data * n)(*data)
    h = C.c_void_p()
    _check(load().mnl_batch_create(n, da, dd, precision, C.c_void_p(stream or 0), C.byref(h)), "mnl_batch_create")
    return h.value


def mnl_batch_num_params(handle: int, count: int):
    offs = (C.c_int64 * count)()
    total = load().mnl_batch_num_params(C.c_void_p(handle), offs)
    return int(total), [int(v) for v in offs]


def mnl_batch_fit(handle: int, opts: mnl_fit_opts | None, theta_ptr: int, count: int):
    probs = (mnl_batch_problem_info * count)()
    info = mnl_batch_info()
    info.problems = probs
    rc = load().mnl_batch_fit(C.c_void_p(handle), C.byref(opts) if opts is not None else None,
                              C.c_void_p(theta_ptr), C.byref(info))
    if rc not in (MNL_OK, MNL_MAXITER) and info.iterations == 0:
        raise MnlError(rc, "mnl_batch_fit")
    return rc, info, [struct_dict(p) for p in probs]


def mnl_batch_destroy(handle: int) -> None:
    _check(load().mnl_batch_destroy(C.c_void_p(handle)), "mnl_batch_destroy")


def mnl_server_opts_default() -> mnl_server_opts:
    o = mnl_server_opts()
    load().mnl_server_opts_default(C.byref(o))
    return o


def mnl_server_create(opts: mnl_server_opts, stream: int | None) -> int:
    h = C.c_void_p()
    _check(load().mnl_server_create(C.byref(opts), C.c_void_p(stream or 0), C.byref(h)), "mnl_server_create")
    return h.value


def mnl_server_submit(handle: int, dims: mnl_dims, host_data: mnl_data, theta0_ptr: int | None) -> int:
    t = C.c_uint64()
    _check(load().mnl_server_submit(C.c_void_p(handle), C.byref(dims), C.byref(host_data),
                                    C.c_void_p(theta0_ptr) if theta0_ptr else None, C.byref(t)), "mnl_server_submit")
    return t.value


def mnl_server_step(handle: int):
    a, q = C.c_int32(), C.c_int32()
    _check(load().mnl_server_step(C.c_void_p(handle), C.byref(a), C.byref(q)), "mnl_server_step")
    return a.value, q.value


def mnl_server_poll(handle: int, ticket: int, theta_ptr: int | None):
    """(finished, result dict or None)."""
    res = mnl_request_result()
    rc = load().mnl_server_poll(C.c_void_p(handle), C.c_uint64(ticket), C.c_void_p(theta_ptr) if theta_ptr else None,
                                C.byref(res))
    if rc == MNL_PENDING:
        return False, None
    _check(rc, "mnl_server_poll")
    return True, struct_dict(res)


def mnl_server_finished(handle: int, cap: int = 4096) -> list[int]:
    buf = (C.c_uint64 * cap)()
    n = C.c_int32()
    _check(load().mnl_server_finished(handle, buf, cap, C.byref(n)), "mnl_server_finished")
    return list(buf[: n.value])


def mnl_server_memory_in_use(handle: int) -> int:
    return int(load().mnl_server_memory_in_use(C.c_void_p(handle)))


def mnl_server_destroy(handle: int) -> None:
    _check(load().mnl_server_destroy(C.c_void_p(handle)), "mnl_server_destroy")
