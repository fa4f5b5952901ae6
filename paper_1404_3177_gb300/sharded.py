"""Observation-sharded Newton-Raphson across processes, one GPU each.

l, g and -H are sums over the observations (Sec. 3.1 eq. "log-lik function",
Sec. 3.3 eqs. "loglik gradient" and "hessian block"), so with the rows split
over ranks one Newton step (eq. "NR update", with the step halving of Sec.
3.1) needs two exchanges:

  1. every rank forms the partial sums [l, sum|l_i|, g, lower(-H)] of its
     rows (mnl_shard_grad_hess); one all-reduce adds them;
  2. every rank solves the same system (mnl_shard_solve; identical summed
     inputs give identical steps, so no broadcast is needed), and each
     line-search trial adds the ranks' partial log-likelihoods at
     theta + t delta (mnl_shard_loglik; an all-reduce of two doubles).

The arithmetic is in the library's kernels; this module only moves the sums
between ranks (torch.distributed: NCCL on GPU tensors, or through host memory
for a CPU backend such as gloo) and takes the same accept / stop decisions as
mnl_newton_step and mnl_fit.  The engine is pluggable: ShardEngine wraps one
rank's handle; anything with the same four methods can stand in for it.
"""
from __future__ import annotations

import math

import torch

from . import _native as nat


class ShardEngine:
    """One rank's observations behind the C ABI (argument marshalling only)."""

    def __init__(self, mnl):
        self.m = mnl
        self.n = mnl.n_theta
        dev = torch.device("cuda", torch.cuda.current_device())
        self.sums = torch.empty(nat.mnl_shard_sums_size(mnl.dims), dtype=torch.float64, device=dev)
        self.delta = torch.empty(self.n, dtype=torch.float64, device=dev)
        self.l2 = torch.empty(2, dtype=torch.float64, device=dev)
        self.roundoff = nat.mnl_loglik_roundoff(mnl.h)
        self.fp64 = mnl.precision == nat.MNL_FP64

    def grad_hess(self, theta):
        nat.mnl_shard_grad_hess(self.m.h, theta.data_ptr(), self.sums.data_ptr())
        return self.sums

    def solve(self, sums):
        info = nat.mnl_shard_solve(self.m.h, sums.data_ptr(), self.delta.data_ptr())
        return self.delta, info

    def loglik(self, theta, delta, t):
        nat.mnl_shard_loglik(self.m.h, theta.data_ptr(), delta.data_ptr() if delta is not None else None, t,
                             self.l2.data_ptr())
        return self.l2


class ShardedNewton:
    """Newton-Raphson over the summed partials of all ranks of `group`."""

    def __init__(self, engine, group=None):
        import torch.distributed as dist
        self.e = engine
        self.dist = dist
        self.group = group
        self.on_device = dist.is_initialized() and dist.get_backend(group) == "nccl"

    def allreduce(self, t):
        """In-place sum over the ranks (bitwise the same result on every rank)."""
        if not self.dist.is_initialized() or self.dist.get_world_size(self.group) == 1:
            return t
        if self.on_device or t.device.type == "cpu":
            self.dist.all_reduce(t, group=self.group)
            return t
        h = t.cpu()
        self.dist.all_reduce(h, group=self.group)
        t.copy_(h)
        return t

    def step(self, theta, gtol=0.0, max_halvings=30):
        """One iteration on theta (updated in place).  Returns a dict; `converged` when max|g| < gtol (theta is
        then unchanged)."""
        n = theta.numel()
        sums = self.allreduce(self.e.grad_hess(theta))
        l0, labs = float(sums[0]), float(sums[1])
        ginf = float(sums[2:2 + n].abs().max())
        if not (math.isfinite(l0) and math.isfinite(ginf)):
            raise nat.MnlError(nat.MNL_ERR_NONFINITE, "ShardedNewton.step")
        out = {"loglik_old": l0, "grad_inf": ginf, "converged": ginf < gtol}
        if out["converged"]:
            out["loglik_new"] = l0
            return out
        delta, sinfo = self.e.solve(sums)
        tau = 8.0 * self.e.roundoff * labs
        t = 1.0
        for j in range(max_halvings + 1):
            lt = float(self.allreduce(self.e.loglik(theta, delta, t))[0])
            if math.isfinite(lt) and lt >= l0 - tau:
                theta.add_(delta, alpha=t)
                out.update(loglik_new=lt, halvings=j, step_scale=t, ls_evals=j + 1,
                           step_inf=t * float(delta.abs().max()), theta_inf=float(theta.abs().max()),
                           solve=sinfo)
                return out
            t *= 0.5
        raise nat.MnlError(nat.MNL_ERR_LINESEARCH, "ShardedNewton.step")

    def fit(self, theta, maxiter=50, gtol=1e-8, steptol=None, max_halvings=30):
        """Newton-Raphson to convergence with mnl_fit's stopping rules (gtol on max|g|, the relative step
        test, and the float32 gradient's noise-floor stop).  theta is updated in place."""
        if steptol is None:
            steptol = 1e-10 if self.e.fp64 else 1e-7
        prev = float("inf")
        iters = 0
        stop = "maxiter"
        info = {}
        for it in range(maxiter):
            info = self.step(theta, gtol=gtol, max_halvings=max_halvings)
            if info["converged"]:
                stop = "gtol"
                break
            iters += 1
            rel = info["step_inf"] / max(1.0, info["theta_inf"])
            if steptol > 0 and rel <= steptol:
                stop = "steptol"
                break
            if not self.e.fp64 and it > 0 and rel > 0.5 * prev and rel <= 1e-5:
                stop = "noise"
                break
            prev = rel
        return {"iters": iters, "stop": stop, "loglik": info.get("loglik_new"), "grad_inf": info.get("grad_inf")}
