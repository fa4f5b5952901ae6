"""Mixed Newton solve with the tensor-core panel factorisation (eq. "NR update").

The float32 factor of F = -H (panels of 128 columns, trailing updates as
3xTF32 tcgen05 tiles) and the inverse of the factor carried along with it only
precondition a float64 iterative refinement, so the step must equal the exact
solution of F delta = g to float64 accuracy:
  * FP64 Hessian (precision "fp64", solve "mixed"): the step against the
    oracle's, np.linalg.solve(F_oracle, g_oracle), to 1e-9 relative;
  * BF16 Hessian: the step of the same handle's Hessian solved by the float64
    Cholesky (solve "fp64"), to 1e-10 relative, with no fallback.
Shapes put n_theta across one to eight panels with ragged last panels
(n mod 128 = 2, 11, 1, 104).  MNL_TC_CHOL_MIN_N = 1 sends these small problems
through the tensor-core factorisation.
"""
import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (N, K, p, d, f): n_theta = (K-1)(p+d) + f
SHAPES = {
    "n130": (3000, 3, 65, 0, 0),     # 2 panels, last one 2 columns wide
    "n267": (5003, 12, 21, 3, 3),    # 3 panels, last 11
    "n641": (6000, 11, 64, 0, 1),    # 6 panels, last 1
    "n1000": (6000, 9, 125, 0, 0),   # 8 panels, last 104
}


@pytest.fixture(scope="module")
def MNL():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300.api import MNL as cls
    return cls


def dev(prob):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a.size else None  # noqa: E731
    return dict(X=t(prob.X), Y=t(prob.Y), Z=t(prob.Z), choice=torch.from_numpy(prob.choice).cuda(), K=prob.K)


def problem(name):
    N, K, p, d, f = SHAPES[name]
    return datagen.make_problem(N, K, p, d, f, 7000 + N, theta_sd=0.3 / np.sqrt(p + d + 1))


def one_step(MNL, prob, prec, solve, monkeypatch, tensor):
    if tensor:
        monkeypatch.setenv("MNL_TC_CHOL_MIN_N", "1")
    else:
        monkeypatch.setenv("MNL_TC_CHOL_MIN_N", "1000000000")
    with MNL(**dev(prob), precision=prec, solve=solve) as m:
        th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
        info = m.newton_step(th)
        return th.cpu().numpy(), info


@pytest.mark.parametrize("name", list(SHAPES))
def test_tensor_core_solve_fp64_hessian_matches_oracle_step(MNL, name, monkeypatch):
    prob = problem(name)
    step, info = one_step(MNL, prob, "fp64", "mixed", monkeypatch, tensor=True)
    assert info["factor_kind"] == 2 and info["solve_mode"] == 2 and info["fallback"] == 0, info
    assert info["halvings"] == 0, info
    l_ref, g_ref = oracle.loglik_grad(prob)
    F_ref = oracle.neg_hessian(prob)
    d_ref = np.linalg.solve(F_ref, g_ref)
    err = np.abs(step - d_ref).max() / np.abs(d_ref).max()
    assert err <= 1e-9, err


@pytest.mark.parametrize("name", ["n267", "n1000"])
def test_tensor_core_solve_matches_fp64_solve_bf16_hessian(MNL, name, monkeypatch):
    prob = problem(name)
    a, ia = one_step(MNL, prob, "bf16", "fp64", monkeypatch, tensor=False)
    b, ib = one_step(MNL, prob, "bf16", "mixed", monkeypatch, tensor=True)
    assert ia["solve_mode"] == 1 and ib["factor_kind"] == 2 and ib["fallback"] == 0 and ib["refine_steps"] >= 1
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max(), np.abs(a - b).max() / np.abs(a).max()


def test_cooperative_and_tensor_core_factors_agree(MNL, monkeypatch):
    """Both factorisations of the mixed solve reach the same float64 step."""
    prob = problem("n641")
    a, ia = one_step(MNL, prob, "tf32", "mixed", monkeypatch, tensor=False)
    b, ib = one_step(MNL, prob, "tf32", "mixed", monkeypatch, tensor=True)
    assert ia["factor_kind"] == 1 and ib["factor_kind"] == 2
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
