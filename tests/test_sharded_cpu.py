"""The sharded Newton driver's exchange on CPU: two gloo ranks on 127.0.0.1,
each with half of the observations, their partial sums formed by the FP64
oracle (a stand-in engine with the same four methods as the GPU engine), the
all-reduces of sharded.ShardedNewton between them.  The summed l, g, -H and
the fitted coefficients must equal the oracle's on the whole problem: the
exchange adds the two halves' sums (eqs. "log-lik function", "loglik
gradient", "hessian block" are sums over observations) and both ranks take
the same steps.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem():
    return datagen.make_problem(3001, 5, 3, 1, 2, 606, theta_sd=0.4)


def half(prob, rank, world):
    lo, hi = prob.N * rank // world, prob.N * (rank + 1) // world
    return datagen.Problem(hi - lo, prob.K, prob.p, prob.d, prob.f, 0, prob.X[lo:hi], prob.Y[lo:hi],
                           prob.Z[lo:hi], prob.choice[lo:hi], prob.theta_true)


class OracleShard:
    """Partial sums of one rank's rows by the FP64 oracle (test stand-in for sharded.ShardEngine)."""

    roundoff = 2.0 ** -53
    fp64 = True

    def __init__(self, prob):
        self.p = prob
        self.n = prob.n_theta

    def grad_hess(self, theta):
        th = theta.numpy()
        l, g = oracle.loglik_grad(self.p, th)
        F = oracle.neg_hessian(self.p, th)
        low = np.concatenate([F[c:, c] for c in range(self.n)])  # packed lower, column by column
        return torch.from_numpy(np.concatenate([[l, -l], g, low]))  # every l_i <= 0: sum |l_i| = -l

    def solve(self, sums):
        s = sums.numpy()
        n = self.n
        F = np.zeros((n, n))
        o = 2 + n
        for c in range(n):
            F[c:, c] = s[o:o + n - c]
            o += n - c
        F = np.tril(F) + np.tril(F, -1).T
        return torch.from_numpy(np.linalg.solve(F, s[2:2 + n])), {}

    def loglik(self, theta, delta, t):
        l = oracle.loglik(self.p, (theta + t * delta).numpy())
        return torch.tensor([l, -l], dtype=torch.float64)


def _rank(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    from paper_1404_3177_gb300.sharded import ShardedNewton
    prob = problem()
    sn = ShardedNewton(OracleShard(half(prob, rank, world)))
    sums = sn.allreduce(sn.e.grad_hess(torch.zeros(prob.n_theta, dtype=torch.float64)).clone())
    theta = torch.zeros(prob.n_theta, dtype=torch.float64)
    for _ in range(4):  # four Newton steps: compared with the oracle's first four iterates
        sn.step(theta)
    np.save(os.path.join(out_dir, f"theta4_{rank}.npy"), theta.numpy())
    info = sn.fit(theta)
    np.save(os.path.join(out_dir, f"sums{rank}.npy"), sums.numpy())
    np.save(os.path.join(out_dir, f"theta{rank}.npy"), theta.numpy())
    with open(os.path.join(out_dir, f"info{rank}.txt"), "w") as fh:
        fh.write(repr(info))
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_whole_problem(tmp_path):
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    prob = problem()
    n = prob.n_theta
    s0, s1 = (np.load(tmp_path / f"sums{r}.npy") for r in range(2))
    assert np.array_equal(s0, s1)  # every rank holds the same sums
    l_ref, g_ref = oracle.loglik_grad(prob)
    F_ref = oracle.neg_hessian(prob)
    assert abs(s0[0] - l_ref) <= 1e-12 * abs(l_ref)
    assert np.abs(s0[2:2 + n] - g_ref).max() <= 1e-11 * np.abs(g_ref).max()
    low = np.concatenate([F_ref[c:, c] for c in range(n)])
    assert np.abs(s0[2 + n:] - low).max() <= 1e-11 * np.abs(low).max()
    a0, a1 = (np.load(tmp_path / f"theta4_{r}.npy") for r in range(2))
    assert np.array_equal(a0, a1)  # both ranks took the same steps
    ref4, st = oracle.fit(prob, maxiter=4, gtol=0.0, steptol=0.0)
    assert st["iters"] == 4
    assert np.abs(a0 - ref4).max() <= 1e-10 * np.abs(ref4).max()
    t0, t1 = (np.load(tmp_path / f"theta{r}.npy") for r in range(2))
    assert np.array_equal(t0, t1)
    ref, _ = oracle.fit(prob)
    assert np.abs(t0 - ref).max() <= 1e-6 * np.abs(ref).max()  # the coefficient bar
    _, g = oracle.loglik_grad(prob, t0)
    assert np.abs(g).max() < 1e-6
