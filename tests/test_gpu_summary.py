"""Standard errors and predicted probabilities on the GPU (the summary and
predict methods of the package, Sec. 2.3) against the FP64 oracle.

  * mnl_std_errors, FP64 mode: sqrt(diag((-H)^-1)) at the oracle's estimate
    against oracle.std_errors (itself pinned to closed forms), 1e-9 relative;
  * BF16 mode: against the same formula applied in float64 by NumPy to the
    handle's own Hessian (the inverse and the column norms, 1e-9), and against
    the oracle within the error that the BF16 Hessian (2e-3) carries into
    (-H)^-1 (bounded here by 10 x 2e-3 x cond(-H));
  * mnl_predict: P and l against oracle.probs, 1e-12 (FP64) and 2e-6 (float32
    pass) absolute.
"""
import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


@pytest.fixture(scope="module")
def fitted():
    # n_theta = 11 * 24 + 3 = 267: five 64-column panels of the float64 factor, the last one ragged
    prob = datagen.make_problem(20011, 12, 21, 3, 3, 515, theta_sd=0.25)
    th, _ = oracle.fit(prob)
    return prob, th, oracle.std_errors(prob, th)


def test_std_errors_fp64_match_the_oracle(MNL, fitted):
    prob, th, se_ref = fitted
    with MNL(**dev(prob), precision="fp64") as m:
        se = m.std_errors(torch.from_numpy(th).cuda()).cpu().numpy()
    assert np.abs(se - se_ref).max() <= 1e-9 * np.abs(se_ref).max(), np.abs(se / se_ref - 1).max()


def test_std_errors_bf16_from_the_handles_hessian(MNL, fitted):
    prob, th, se_ref = fitted
    tht = torch.from_numpy(th).cuda()
    with MNL(**dev(prob), precision="bf16") as m:
        se = m.std_errors(tht).cpu().numpy()
        H = m.hessian(tht).cpu().numpy()
    se_own = np.sqrt(np.diag(np.linalg.inv(-H)))
    assert np.abs(se - se_own).max() <= 1e-9 * se_own.max()
    F_ref = oracle.neg_hessian(prob, th)
    bound = 10 * 2e-3 * np.linalg.cond(F_ref)
    assert np.abs(se / se_ref - 1).max() <= bound, (np.abs(se / se_ref - 1).max(), bound)


def test_std_errors_report_a_singular_design(MNL):
    from paper_1404_3177_gb300._native import MnlError, MNL_ERR_NOT_PD
    prob = datagen.make_problem(500, 4, 3, 0, 0, 3)
    prob.X[:, 2] = 0.0
    with MNL(**dev(prob), precision="fp64") as m:
        with pytest.raises(MnlError) as e:
            m.std_errors(None)
        assert e.value.status == MNL_ERR_NOT_PD


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16", 2e-6)])
def test_predict_matches_oracle_probabilities(MNL, fitted, prec, tol):
    prob, th, _ = fitted
    P_ref, l_ref = oracle.probs(prob, th)
    with MNL(**dev(prob), precision=prec) as m:
        P, l = m.predict(torch.from_numpy(th).cuda())
    P = P.cpu().numpy()
    assert np.abs(P - P_ref).max() <= tol
    assert abs(l - l_ref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(l_ref)


def test_predict_for_new_data(MNL, fitted):
    """The package's predict with new data: a handle on other observations, the same coefficients."""
    prob, th, _ = fitted
    new = datagen.make_problem(3001, prob.K, prob.p, prob.d, prob.f, 616, theta_true=prob.theta_true)
    P_ref, _ = oracle.probs(new, th)
    with MNL(**dev(new), precision="fp64") as m:
        P, _ = m.predict(torch.from_numpy(th).cuda())
    assert np.abs(P.cpu().numpy() - P_ref).max() <= 1e-12
