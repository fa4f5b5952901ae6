"""Observation weights and the paper-literal gamma_0 (gamma_base = 1) on the
GPU path, against the FP64 oracle (whose weights are pinned in
test_oracle_weights.py and whose gamma_base = 1 form in test_oracle_pins.py).

Tolerances as in test_gpu_parity.py: l relative 1e-12 / 1e-6, g normwise
1e-11 / 1e-6, -H relative Frobenius 1e-10 / 2e-3 (FP64 / float32 pass with
tensor-core Hessian), converged coefficients 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRECS = ["fp64", "tf32", "bf16"]
TOL = {"fp64": dict(l=1e-12, g=1e-11, H=1e-10), "tf32": dict(l=1e-6, g=1e-6, H=2e-3),
       "bf16": dict(l=1e-6, g=1e-6, H=2e-3)}


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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def weights(N, seed):
    w = np.random.default_rng(seed).uniform(0.0, 3.0, N).astype(np.float32)
    w[::10] = 0.0
    return w


def check(api, prob, prec, th, **kw):
    tol = TOL[prec]
    l_ref, g_ref = oracle.loglik_grad(prob, th)
    F_ref = oracle.neg_hessian(prob, th)
    with api.MNL(**dev(prob), precision=prec, **kw) as m:
        tht = torch.from_numpy(th).cuda()
        l, g = m.loglik_grad(tht)
        H = m.hessian(tht).cpu().numpy()
    assert abs(l - l_ref) <= tol["l"] * abs(l_ref), (prec, l, l_ref)
    assert rel(g.cpu().numpy(), g_ref) <= tol["g"], prec
    assert rel(-H, F_ref) <= tol["H"], (prec, rel(-H, F_ref))


@pytest.mark.parametrize("prec", PRECS)
def test_weighted_l_g_H_match_oracle(lib, prec):
    nat, api = lib
    prob = datagen.make_problem(5003, 12, 21, 3, 3, 71, theta_sd=0.25)
    prob.w = weights(prob.N, 1)
    th = np.random.default_rng(2).normal(0, 0.1, prob.n_theta)
    check(api, prob, prec, th, weights=torch.from_numpy(prob.w).cuda())


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_weighted_wide_shape_matches_oracle(lib, prec):
    """The wide tiled pass (beta gradient in its own kernel) with weights."""
    nat, api = lib
    prob = datagen.make_problem(3001, 70, 40, 0, 8, 72, theta_sd=0.05)
    prob.w = weights(prob.N, 3)
    th = np.random.default_rng(4).normal(0, 0.02, prob.n_theta)
    l_ref, g_ref = oracle.loglik_grad(prob, th)
    with api.MNL(**dev(prob), precision=prec, weights=torch.from_numpy(prob.w).cuda()) as m:
        l, g = m.loglik_grad(torch.from_numpy(th).cuda())
    assert abs(l - l_ref) <= TOL[prec]["l"] * abs(l_ref)
    assert rel(g.cpu().numpy(), g_ref) <= TOL[prec]["g"]


@pytest.mark.parametrize("prec", PRECS)
def test_weighted_fit_matches_oracle_fit(lib, prec):
    nat, api = lib
    prob = datagen.make_problem(6000, 5, 4, 1, 2, 73, theta_sd=0.4)
    prob.w = weights(prob.N, 5)
    ref, _ = oracle.fit(prob)
    with api.MNL(**dev(prob), precision=prec, weights=torch.from_numpy(prob.w).cuda()) as m:
        th, info = m.fit()
    assert info["status"] == 0, info
    assert np.abs(th.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()


def test_integer_weights_equal_repeated_rows(lib):
    nat, api = lib
    prob = datagen.make_problem(3000, 6, 5, 2, 1, 74, theta_sd=0.3)
    w = np.random.default_rng(6).integers(0, 4, prob.N)
    idx = np.repeat(np.arange(prob.N), w)
    rep = datagen.Problem(len(idx), prob.K, prob.p, prob.d, prob.f, 0, prob.X[idx], prob.Y[idx], prob.Z[idx],
                          prob.choice[idx], prob.theta_true)
    th = torch.from_numpy(np.random.default_rng(7).normal(0, 0.1, prob.n_theta)).cuda()
    with api.MNL(**dev(prob), precision="fp64", weights=torch.from_numpy(w.astype(np.float32)).cuda()) as m:
        lw, gw = m.loglik_grad(th)
        Hw = m.hessian(th).cpu().numpy()
    with api.MNL(**dev(rep), precision="fp64") as m:
        lr, gr = m.loglik_grad(th)
        Hr = m.hessian(th).cpu().numpy()
    assert abs(lw - lr) <= 1e-12 * abs(lr)
    assert rel(gw.cpu().numpy(), gr.cpu().numpy()) <= 1e-11
    assert rel(Hw, Hr) <= 1e-11


def test_invalid_weights_are_rejected(lib):
    nat, api = lib
    prob = datagen.make_problem(500, 3, 2, 0, 0, 75)
    with api.MNL(**dev(prob), precision="bf16") as m:
        for bad, code in ((-1.0, nat.MNL_ERR_INVALID_ARG), (float("nan"), nat.MNL_ERR_NONFINITE)):
            w = torch.ones(prob.N, dtype=torch.float32, device="cuda")
            w[17] = bad
            with pytest.raises(nat.MnlError) as e:
                m.set_weights(w)
            assert e.value.status == code


# ---------------------------------------------------------------------------
# gamma_base = 1 (gamma_0 estimated, eq. "theta vec")
# ---------------------------------------------------------------------------

def gb1_problem(N=4001, K=6, p=3, d=2, f=2, seed=81):
    return datagen.make_problem(N, K, p, d, f, seed, theta_sd=0.3, gamma_base=1)


@pytest.mark.parametrize("prec", PRECS)
def test_gamma0_l_g_H_match_oracle(lib, prec):
    nat, api = lib
    prob = gb1_problem()
    assert prob.n_theta == (prob.K - 1) * prob.p + prob.K * prob.d + prob.f
    th = np.random.default_rng(9).normal(0, 0.2, prob.n_theta)
    check(api, prob, prec, th, gamma_base=1)


@pytest.mark.parametrize("prec", PRECS)
def test_gamma0_fit_matches_oracle_fit(lib, prec):
    nat, api = lib
    prob = gb1_problem(6000, 4, 2, 2, 1, 82)
    ref, _ = oracle.fit(prob)
    with api.MNL(**dev(prob), precision=prec, gamma_base=1) as m:
        th, info = m.fit()
    assert info["status"] == 0, info
    assert np.abs(th.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()


def test_gamma0_with_weights_std_errors_and_predict(lib):
    nat, api = lib
    prob = gb1_problem(5000, 5, 3, 2, 2, 83)
    prob.w = weights(prob.N, 8)
    ref, _ = oracle.fit(prob)
    se_ref = oracle.std_errors(prob, ref)
    P_ref, l_ref = oracle.probs(prob, ref)
    with api.MNL(**dev(prob), precision="fp64", gamma_base=1, weights=torch.from_numpy(prob.w).cuda()) as m:
        th, info = m.fit()
        se = m.std_errors(torch.from_numpy(ref).cuda()).cpu().numpy()
        P, l = m.predict(torch.from_numpy(ref).cuda())
    assert np.abs(th.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    assert np.abs(se - se_ref).max() <= 1e-9 * np.abs(se_ref).max()
    assert np.abs(P.cpu().numpy() - P_ref).max() <= 1e-12 and abs(l - l_ref) <= 1e-12 * abs(l_ref)


@pytest.mark.parametrize("d,f,n_p", [(50, 0, 5000), (45, 5, 4505)])
def test_table1_problem_shapes_with_gamma0(lib, d, f, n_p):
    """The paper's Table 1 problems Y (50 alternative-specific variables with per-alternative coefficients,
    n_p = 5000) and YZ (45 + 5 generic, n_p = 4505) at K = 100, on a small N."""
    nat, api = lib
    prob = datagen.make_problem(2003, 100, 0, d, f, 84, intercept=False, theta_sd=0.02, gamma_base=1)
    assert prob.n_theta == n_p
    th = np.random.default_rng(10).normal(0, 0.02, prob.n_theta)
    l_ref, g_ref = oracle.loglik_grad(prob, th)
    with api.MNL(**dev(prob), precision="bf16", gamma_base=1) as m:
        assert m.n_theta == n_p
        l, g = m.loglik_grad(torch.from_numpy(th).cuda())
    assert abs(l - l_ref) <= 1e-6 * abs(l_ref)
    assert rel(g.cpu().numpy(), g_ref) <= 1e-6
