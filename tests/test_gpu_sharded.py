"""Observation sharding through the C ABI: two ranks (processes, gloo through
host memory) on one GPU, each with half of the observations.  No kernel of one
rank waits on the other: the ranks meet only in host-side all-reduces between
calls.  The summed l, g and -H must match the FP64 oracle on the whole problem
at the single-GPU tolerances, and so must the fitted coefficients.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = {"fp64": dict(l=1e-12, g=1e-11, H=1e-10), "bf16": dict(l=1e-6, g=1e-6, H=2e-3)}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem():
    # n_theta = 11 * 24 + 3 = 267, N odd so the halves differ in size
    return datagen.make_problem(8001, 12, 21, 3, 3, 717, theta_sd=0.25)


def _rank(rank, world, port, out_dir, prec):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300.api import MNL
    from paper_1404_3177_gb300.sharded import ShardEngine, ShardedNewton
    prob = problem()
    lo, hi = prob.N * rank // world, prob.N * (rank + 1) // world
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a[lo:hi])).cuda()  # noqa: E731
    with MNL(X=t(prob.X), Y=t(prob.Y), Z=t(prob.Z), choice=t(prob.choice), K=prob.K, precision=prec) as m:
        sn = ShardedNewton(ShardEngine(m))
        theta = torch.zeros(prob.n_theta, dtype=torch.float64, device="cuda")
        sums = sn.allreduce(sn.e.grad_hess(theta)).cpu().numpy()
        info = sn.fit(theta)
        np.save(os.path.join(out_dir, f"sums{rank}.npy"), sums)
        np.save(os.path.join(out_dir, f"theta{rank}.npy"), theta.cpu().numpy())
        with open(os.path.join(out_dir, f"info{rank}.txt"), "w") as fh:
            fh.write(repr(info))
    dist.destroy_process_group()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_two_ranks_on_halves_match_the_whole_problem(prec, tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path), prec), nprocs=2, join=True)
    prob = problem()
    n = prob.n_theta
    tol = TOL[prec]
    s0, s1 = (np.load(tmp_path / f"sums{r}.npy") for r in range(2))
    assert np.array_equal(s0, s1)
    l_ref, g_ref = oracle.loglik_grad(prob)
    F_ref = oracle.neg_hessian(prob)
    assert abs(s0[0] - l_ref) <= tol["l"] * abs(l_ref)
    assert np.linalg.norm(s0[2:2 + n] - g_ref) <= tol["g"] * np.linalg.norm(g_ref)
    F = np.zeros((n, n))
    o = 2 + n
    for c in range(n):
        F[c:, c] = s0[o:o + n - c]
        o += n - c
    F = np.tril(F) + np.tril(F, -1).T
    assert np.linalg.norm(F - F_ref) <= tol["H"] * np.linalg.norm(F_ref)
    t0, t1 = (np.load(tmp_path / f"theta{r}.npy") for r in range(2))
    assert np.array_equal(t0, t1)
    ref, _ = oracle.fit(prob)
    assert np.abs(t0 - ref).max() <= 1e-6 * np.abs(ref).max()
