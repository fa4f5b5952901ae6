"""Bounded device waits: every wait of the pipelined kernels gives up after a
host-settable bound (mnl_set_wait_bound), the call returns MNL_ERR_TIMEOUT
with the kernels that gave up named in mnl_step_info.wait_errors, and the
handle and the GPU stay usable.

A bound of 1 ns makes a wait run out whenever what it waits for is not
already complete at its first check: the tensor-core pipelines (TMA stages,
accumulators) and the grid barriers of the factorisations always wait, so
they always time out; the pass's tile copies are issued well ahead of their
use and have usually landed by then, so its wait is exercised but may not run
out.  Copies and tensor-core operations already issued are still waited for
with the default bound before a block exits, so nothing is left in flight.  Nothing here faults
or hangs: every wait is bounded.  Afterwards the same handle with the default
bound, and a fresh handle, match the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300 import _native, api
    return _native, api


def dev(prob):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a.size else None  # noqa: E731
    return dict(X=t(prob.X), Y=t(prob.Y), Z=t(prob.Z), choice=torch.from_numpy(prob.choice).cuda(), K=prob.K)


def _timed_out_step(nat, m):
    th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
    nat.mnl_set_wait_bound(m.h, 1)
    with pytest.raises(nat.MnlError) as e:
        m.newton_step(th)
    assert e.value.status == nat.MNL_ERR_TIMEOUT
    assert float(th.abs().max()) == 0.0  # theta untouched
    return e.value.info["wait_errors"]


@pytest.mark.parametrize("tensor_factor", [False, True])
def test_every_bounded_kernel_times_out_and_the_handle_recovers(lib, tensor_factor, monkeypatch):
    nat, api = lib
    monkeypatch.setenv("MNL_TC_CHOL_MIN_N", "1" if tensor_factor else "1000000000")
    prob = datagen.make_problem(5003, 12, 21, 3, 3, 4321, theta_sd=0.25)  # tiled pass, tcgen05 Z and class blocks
    with api.MNL(**dev(prob), precision="bf16") as m:
        bits = _timed_out_step(nat, m)
        assert bits & nat.MNL_WAIT_SYRK, bits
        assert bits & (nat.MNL_WAIT_PANEL if tensor_factor else nat.MNL_WAIT_COOP), bits
        # default bounds again: the same handle gives the oracle's l, g and a full step
        nat.mnl_set_wait_bound(m.h, 0)
        l, g = m.loglik_grad()
        th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
        info = m.newton_step(th)
        assert info["wait_errors"] == 0 and info["loglik_new"] > info["loglik_old"]
    l_ref, g_ref = oracle.loglik_grad(prob)
    assert abs(l - l_ref) <= 1e-6 * abs(l_ref)
    assert np.linalg.norm(g.cpu().numpy() - g_ref) <= 1e-6 * np.linalg.norm(g_ref)


def test_fp64_factor_barrier_times_out_and_a_fresh_handle_matches_the_oracle(lib):
    nat, api = lib
    prob = datagen.make_problem(3001, 7, 5, 2, 2, 99, theta_sd=0.3)
    with api.MNL(**dev(prob), precision="fp64") as m:
        bits = _timed_out_step(nat, m)
        assert bits & nat.MNL_WAIT_COOP, bits
    with api.MNL(**dev(prob), precision="fp64") as m:
        l, g = m.loglik_grad()
        H = m.hessian().cpu().numpy()
    l_ref, g_ref = oracle.loglik_grad(prob)
    F_ref = oracle.neg_hessian(prob)
    assert abs(l - l_ref) <= 1e-12 * abs(l_ref)
    assert np.linalg.norm(g.cpu().numpy() - g_ref) <= 1e-11 * np.linalg.norm(g_ref)
    assert np.linalg.norm(-H - F_ref) <= 1e-10 * np.linalg.norm(F_ref)
