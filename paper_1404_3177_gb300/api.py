"""torch-facing wrapper around the C ABI (marshalling only; no arithmetic here)."""
from __future__ import annotations

import numpy as np
import torch

from . import _native as nat


def _ptr(t):
    return t.data_ptr() if t is not None and t.numel() > 0 else None


class MNL:
    """One multinomial-logit problem resident on the current CUDA device.

    X [N][p], Y [N][K][d], Z [N][K][f] (float32) and choice [N] (int32) are CUDA
    tensors that must outlive this object; pass None for an empty block.  K is
    taken from Y or Z, or must be given.  ``precision`` is "fp64", "tf32" or
    "bf16" (the arithmetic of the Hessian contraction, see include/mnl.h).
    """

    def __init__(self, X=None, Y=None, Z=None, choice=None, *, K=None, precision="bf16", stream=None,
                 host_owned_dims=None, solve="auto", gamma_base=0, weights=None, truncated=False):
        self.precision = nat.PRECISIONS[precision]
        self._stream = (stream or torch.cuda.current_stream()).cuda_stream
        if host_owned_dims is not None:
            self.dims = host_owned_dims
            self._keep = ()
            self.h = nat.mnl_create(self.dims, None, self.precision, self._stream)
            nat.mnl_set_solve(self.h, nat.SOLVES[solve])
            return
        if choice is None:
            raise ValueError("choice is required")
        N = choice.shape[0]
        if Y is not None:
            K = Y.shape[1]
        elif Z is not None:
            K = Z.shape[1]
        if K is None:
            raise ValueError("K must be given when neither Y nor Z is present")
        p = X.shape[1] if X is not None else 0
        d = Y.shape[2] if Y is not None else 0
        f = Z.shape[2] if Z is not None else 0
        for name, t, dt in (("X", X, torch.float32), ("Y", Y, torch.float32), ("Z", Z, torch.float32),
                            ("choice", choice, torch.int32)):
            if t is not None and (not t.is_cuda or t.dtype != dt or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {dt}")
        self._keep = (X, Y, Z, choice)
        self.dims = nat.mnl_dims(N, K, p, d, f, gamma_base)
        data = nat.mnl_data(_ptr(X), _ptr(Y), _ptr(Z), _ptr(choice))
        self.h = nat.mnl_create_ex(self.dims, data, self.precision, nat.MNL_CREATE_TRUNCATED if truncated else 0,
                                   self._stream)
        nat.mnl_set_solve(self.h, nat.SOLVES[solve])
        if weights is not None:
            self.set_weights(weights)

    def set_weights(self, w):
        """Observation (case) weights: a contiguous float32 CUDA tensor [N], or None."""
        if w is not None and (not w.is_cuda or w.dtype != torch.float32 or not w.is_contiguous()):
            raise ValueError("weights must be a contiguous float32 CUDA tensor")
        self._w = w
        nat.mnl_set_weights(self.h, _ptr(w))

    @classmethod
    def with_host_upload(cls, N, K, p, d, f, *, precision="bf16", stream=None, solve="auto"):
        """A handle that owns its device copies of the data; fill it with ``upload``."""
        return cls(precision=precision, stream=stream, host_owned_dims=nat.mnl_dims(N, K, p, d, f, 0), solve=solve)

    def upload(self, X=None, Y=None, Z=None, choice=None):
        """Copy host tensors (pinned for speed) into the handle's own device buffers."""
        data = nat.mnl_data(_ptr(X), _ptr(Y), _ptr(Z), _ptr(choice))
        self._host_keep = (X, Y, Z, choice)
        nat.mnl_upload(self.h, data)

    @property
    def n_theta(self) -> int:
        return nat.mnl_num_params(self.dims)

    def _theta(self, theta):
        if theta is None:
            return torch.zeros(self.n_theta, dtype=torch.float64, device="cuda")
        if not theta.is_cuda or theta.dtype != torch.float64 or theta.shape != (self.n_theta,):
            raise ValueError("theta must be a float64 CUDA tensor of shape (n_theta,)")
        return theta.contiguous()

    def loglik_grad(self, theta=None, grad=True):
        th = self._theta(theta)
        g = torch.empty(self.n_theta, dtype=torch.float64, device=th.device) if grad else None
        l = nat.mnl_loglik_grad(self.h, th.data_ptr(), True, _ptr(g))
        return l, g

    def hessian(self, theta=None):
        """Hessian (paper sign, negative definite), float64 [n][n] (symmetric)."""
        th = self._theta(theta)
        H = torch.empty(self.n_theta, self.n_theta, dtype=torch.float64, device=th.device)
        nat.mnl_hessian(self.h, th.data_ptr(), H.data_ptr())
        return H

    def hessian_vec(self, theta, v):
        """H v at theta (paper sign), float64 [n_theta] (CUDA), without forming H."""
        th = self._theta(theta)
        vv = self._theta(v)
        out = torch.empty(self.n_theta, dtype=torch.float64, device=th.device)
        nat.mnl_hessian_vec(self.h, th.data_ptr(), vv.data_ptr(), out.data_ptr())
        return out

    def std_errors(self, theta):
        """Standard errors sqrt(diag((-H)^-1)) at theta, float64 [n_theta] (CUDA)."""
        th = self._theta(theta)
        se = torch.empty(self.n_theta, dtype=torch.float64, device=th.device)
        nat.mnl_std_errors(self.h, th.data_ptr(), se.data_ptr())
        return se

    def predict(self, theta):
        """(choice probabilities float64 [N][K] (CUDA), l(theta))."""
        th = self._theta(theta)
        P = torch.empty(self.dims.N, self.dims.K, dtype=torch.float64, device=th.device)
        l = nat.mnl_predict(self.h, th.data_ptr(), P.data_ptr())
        return P, l

    def check_collinear(self, tol=1e-6):
        """Flags (numpy int32 [p + K d + f]: X | Y_0..Y_{K-1} | Z) of the data columns that depend on earlier
        ones (Sec. 2.3 linDepTol, App. B); see mnl_check_collinear."""
        d = self.dims
        flags, _ = nat.mnl_check_collinear(self.h, tol, d.p + d.K * d.d + d.f)
        return np.asarray(flags, dtype=np.int32)

    def drop_columns(self, flags):
        """Hold the coefficients of the flagged columns at their current values (None: the full model)."""
        nat.mnl_drop_columns(self.h, None if flags is None else [int(x) for x in flags])

    def newton_step(self, theta):
        """One Newton-Raphson iteration; theta (float64 CUDA) is updated in place."""
        info = nat.mnl_newton_step(self.h, self._theta(theta).data_ptr())
        return nat.struct_dict(info)

    def fit(self, theta0=None, **opts):
        o = nat.mnl_fit_opts_default()
        for k, v in opts.items():
            setattr(o, k, v)
        th = self._theta(theta0).clone() if theta0 is not None else self._theta(None)
        info = nat.mnl_fit(self.h, o, th.data_ptr())
        return th, nat.struct_dict(info)

    def close(self):
        if getattr(self, "h", None):
            nat.mnl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class MNLBatch:
    """Many independent problems fitted together (one grouped launch per Newton phase).

    ``problems`` is a list of dicts with CUDA tensors X, Y, Z, choice (None for
    an empty block) and K; they must outlive this object.
    """

    def __init__(self, problems, *, precision="bf16", stream=None):
        self.precision = nat.PRECISIONS[precision]
        self._stream = (stream or torch.cuda.current_stream()).cuda_stream
        dims, data, keep = [], [], []
        for pr in problems:
            X, Y, Z, c = pr.get("X"), pr.get("Y"), pr.get("Z"), pr["choice"]
            K = Y.shape[1] if Y is not None else Z.shape[1] if Z is not None else pr["K"]
            dims.append(nat.mnl_dims(c.shape[0], K, X.shape[1] if X is not None else 0,
                                     Y.shape[2] if Y is not None else 0, Z.shape[2] if Z is not None else 0, 0))
            data.append(nat.mnl_data(_ptr(X), _ptr(Y), _ptr(Z), _ptr(c)))
            keep.append((X, Y, Z, c))
        self._keep = keep
        self.count = len(dims)
        self.h = nat.mnl_batch_create(dims, data, self.precision, self._stream)
        self.n_total, self.offsets = nat.mnl_batch_num_params(self.h, self.count)
        self.sizes = [nat.mnl_num_params(d) for d in dims]

    def fit(self, theta0=None, **opts):
        """Returns (packed float64 theta, summary dict, per-problem dicts, status)."""
        o = nat.mnl_fit_opts_default()
        for k, v in opts.items():
            setattr(o, k, v)
        th = torch.zeros(self.n_total, dtype=torch.float64, device="cuda") if theta0 is None else theta0.clone()
        rc, info, per = nat.mnl_batch_fit(self.h, o, th.data_ptr(), self.count)
        summary = {k: getattr(info, k) for k, _ in info._fields_ if k != "problems"}
        return th, summary, per, rc

    def split(self, theta):
        return [theta[o:o + n] for o, n in zip(self.offsets, self.sizes)]

    def close(self):
        if getattr(self, "h", None):
            nat.mnl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class MNLServer:
    """Continuous batching of fit requests (one Newton iteration of every admitted request per step)."""

    def __init__(self, *, precision="bf16", mem_budget=80 << 30, max_active=4096, max_skips=8, stream=None, **fit):
        o = nat.mnl_server_opts_default()
        o.mem_budget = int(mem_budget)
        o.precision = nat.PRECISIONS[precision]
        o.max_active = max_active
        o.max_skips = max_skips
        for k, v in fit.items():
            setattr(o.fit, k, v)
        self.h = nat.mnl_server_create(o, (stream or torch.cuda.current_stream()).cuda_stream)
        self._sizes = {}

    def submit(self, X=None, Y=None, Z=None, choice=None, K=None, theta0=None):
        """X, Y, Z, choice: numpy arrays (float32 / int32) on the host; returns a ticket."""
        N = choice.shape[0]
        if Y is not None and Y.size:
            K = Y.shape[1]
        elif Z is not None and Z.size:
            K = Z.shape[1]
        p = X.shape[1] if X is not None else 0
        d = Y.shape[2] if Y is not None and Y.size else 0
        f = Z.shape[2] if Z is not None and Z.size else 0
        arrs = [np.ascontiguousarray(a) if a is not None else None for a in (X, Y, Z)]
        c = np.ascontiguousarray(choice, dtype=np.int32)
        ptr = lambda a: a.ctypes.data if a is not None and a.size else None  # noqa: E731
        dims = nat.mnl_dims(N, K, p, d, f, 0)
        data = nat.mnl_data(ptr(arrs[0]), ptr(arrs[1]), ptr(arrs[2]), c.ctypes.data)
        th = np.ascontiguousarray(theta0, dtype=np.float64) if theta0 is not None else None
        t = nat.mnl_server_submit(self.h, dims, data, th.ctypes.data if th is not None else None)
        self._sizes[t] = nat.mnl_num_params(dims)
        return t

    def step(self):
        return nat.mnl_server_step(self.h)

    def poll(self, ticket):
        """(theta numpy array, result dict) once finished, else None."""
        out = np.empty(self._sizes[ticket])
        done, res = nat.mnl_server_poll(self.h, ticket, out.ctypes.data)
        if not done:
            return None
        del self._sizes[ticket]
        return out, res

    def finished(self):
        """(ticket, result dict) of every request that finished since the last call (theta: poll it first)."""
        out = []
        while True:
            ts = nat.mnl_server_finished(self.h)
            for t in ts:
                r = self.poll(t)
                out.append((t, r[1]))
            if len(ts) < 4096:
                return out

    def memory_in_use(self):
        return nat.mnl_server_memory_in_use(self.h)

    def close(self):
        if getattr(self, "h", None):
            nat.mnl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
