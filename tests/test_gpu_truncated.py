"""Hessian-free (truncated Newton) path: Hessian-vector products against the
FP64 oracle's -H applied to v, and truncated-Newton fits against the oracle's
fits (the inexact Newton of the paper's closing discussion).

  * mnl_hessian_vec: relative error of H v (2-norm) 1e-12 (FP64), 1e-6
    (float32 pass), on a general shape (X, Y, Z), on the wide shape whose beta
    products run in their own kernel, with weights, and with gamma_base = 1;
  * fits of MNL_CREATE_TRUNCATED handles: coefficients within 1e-6 of the
    oracle's fit; the handle refuses mnl_hessian and holds far less memory;
  * n_theta = 12672 (K = 100, p = 128): a fit whose oracle Hessian would take
    hours; stationarity is checked with the oracle's gradient at the result.
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = {
    "general": lambda: datagen.make_problem(5003, 12, 21, 3, 3, 901, theta_sd=0.25),
    "wide": lambda: datagen.make_problem(3001, 70, 40, 0, 8, 902, theta_sd=0.05),
    "gamma0": lambda: datagen.make_problem(4001, 6, 3, 2, 2, 903, theta_sd=0.3, gamma_base=1),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16", 1e-6)])
def test_hessian_vector_product_matches_oracle(lib, case, prec, tol):
    nat, api = lib
    prob = CASES[case]()
    rng = np.random.default_rng(11)
    th = rng.normal(0, 0.05, prob.n_theta)
    v = rng.normal(0, 1.0, prob.n_theta)
    Hv_ref = -oracle.neg_hessian(prob, th) @ v
    kw = {"gamma_base": 1} if prob.gamma_base else {}
    with api.MNL(**dev(prob), precision=prec, truncated=(case == "wide"), **kw) as m:
        Hv = m.hessian_vec(torch.from_numpy(th).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
    assert rel(Hv, Hv_ref) <= tol, rel(Hv, Hv_ref)


def test_hessian_vector_product_with_weights(lib):
    nat, api = lib
    prob = CASES["general"]()
    prob.w = np.random.default_rng(12).uniform(0, 2, prob.N).astype(np.float32)
    rng = np.random.default_rng(13)
    th, v = rng.normal(0, 0.05, prob.n_theta), rng.normal(0, 1.0, prob.n_theta)
    Hv_ref = -oracle.neg_hessian(prob, th) @ v
    with api.MNL(**dev(prob), precision="fp64", weights=torch.from_numpy(prob.w).cuda()) as m:
        Hv = m.hessian_vec(torch.from_numpy(th).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
    assert rel(Hv, Hv_ref) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16"])
def test_truncated_newton_fit_matches_oracle_fit(lib, prec):
    nat, api = lib
    prob = datagen.make_problem(8000, 8, 6, 2, 2, 904, theta_sd=0.3)
    ref, _ = oracle.fit(prob)
    with api.MNL(**dev(prob), precision=prec, truncated=True) as m:
        th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
        info = m.newton_step(th)
        assert info["cg_iters"] >= 1 and info["factor_kind"] == 0 and info["loglik_new"] > info["loglik_old"]
        th, finfo = m.fit()
        with pytest.raises(nat.MnlError) as e:
            m.hessian()
        assert e.value.status == nat.MNL_ERR_UNSUPPORTED
    assert finfo["status"] == 0, finfo
    assert np.abs(th.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()


def test_truncated_handle_holds_no_hessian(lib):
    nat, api = lib
    prob = datagen.make_problem(20000, 50, 60, 0, 2, 905, theta_sd=0.05)
    d = dev(prob)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    full = api.MNL(**d, precision="bf16")
    torch.cuda.synchronize()
    used_full = free0 - torch.cuda.mem_get_info()[0]
    full.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    tn = api.MNL(**d, precision="bf16", truncated=True)
    torch.cuda.synchronize()
    used_tn = free0 - torch.cuda.mem_get_info()[0]
    tn.close()
    assert used_tn * 4 < used_full, (used_tn, used_full)


def test_truncated_newton_beyond_ten_thousand_coefficients(lib):
    nat, api = lib
    prob = datagen.make_problem(20011, 100, 128, 0, 0, 906, intercept=False, theta_sd=0.02)
    assert prob.n_theta == 12672
    with api.MNL(**dev(prob), precision="fp64", truncated=True) as m:
        th, info = m.fit(gtol=1e-6)
    assert info["status"] == 0 and info["stop_reason"] in (1, 3), info
    _, g = oracle.loglik_grad(prob, th.cpu().numpy())
    l0, g0 = oracle.loglik_grad(prob)
    assert np.abs(g).max() <= 1e-6 * np.abs(g0).max() + 1e-6, np.abs(g).max()
