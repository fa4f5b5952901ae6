"""GPU path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (the stated bars):
  log-likelihood, relative:           1e-12 (FP64)   1e-6 (TF32/BF16: float32 pass, compensated sums)
  gradient, ||dg||_2 / ||g||_2:       1e-11 (FP64)   1e-6
  negative Hessian, rel. Frobenius:   1e-10 (FP64)   2e-3 (tensor-core contraction)
  converged coefficients, max|dtheta| / max|theta|: 1e-6 in every mode.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRECS = ["fp64", "tf32", "bf16"]
TOL = {
    "fp64": dict(l=1e-12, g=1e-11, H=1e-10),
    "tf32": dict(l=1e-6, g=1e-6, H=2e-3),
    "bf16": dict(l=1e-6, g=1e-6, H=2e-3),
}
THETA_TOL = 1e-6
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="session")
def MNL():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300.api import MNL as cls
    return cls


def dev(prob):
    d = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d) if a.size else None  # noqa: E731
    return dict(X=t(prob.X), Y=t(prob.Y), Z=t(prob.Z), choice=torch.from_numpy(prob.choice).to(d), K=prob.K)


def th_dev(theta):
    return torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_lgH(MNL, prob, prec, theta=None, hessian=True):
    tol = TOL[prec]
    th = np.zeros(prob.n_theta) if theta is None else theta
    l_ref, g_ref = oracle.loglik_grad(prob, th)
    with MNL(**dev(prob), precision=prec) as m:
        l, g = m.loglik_grad(th_dev(th))
        g = g.cpu().numpy()
        assert abs(l - l_ref) <= tol["l"] * abs(l_ref), (prec, l, l_ref)
        assert rel(g, g_ref) <= tol["g"], (prec, rel(g, g_ref))
        if hessian:
            F_ref = oracle.neg_hessian(prob, th)
            H = m.hessian(th_dev(th)).cpu().numpy()
            assert np.array_equal(H, H.T)
            assert rel(-H, F_ref) <= tol["H"], (prec, rel(-H, F_ref))
    return True


# A problem spanning three 128-wide Hessian tiles with ragged edges in N and in the columns.
def s1(seed=11):
    return datagen.make_problem(5003, 12, 21, 3, 3, seed, theta_sd=0.25)


@pytest.mark.parametrize("prec", PRECS)
def test_loglik_grad_hessian_at_zero_and_random_theta(MNL, prec):
    prob = s1()
    check_lgH(MNL, prob, prec)
    th = np.random.default_rng(5).normal(0, 0.2, prob.n_theta)
    check_lgH(MNL, prob, prec, th)


EDGE_SHAPES = [
    # (N, K, p, d, f, intercept)
    (4001, 2, 3, 0, 0, True),     # binary logit
    (3000, 5, 1, 0, 0, True),     # intercept only
    (2500, 6, 0, 0, 3, False),    # generic coefficients only (no class blocks)
    (2999, 40, 4, 2, 1, True),    # K > 32: two alternatives per lane
    (3001, 100, 3, 0, 2, True),   # K = 100
    (1, 3, 2, 1, 1, True),        # a single observation
    (7, 4, 2, 1, 2, True),        # fewer observations than one tile
    (1500, 3, 150, 0, 0, True),   # q > 128: a class block spans three tiles
    (2000, 9, 7, 0, 0, False),    # X only, no intercept
    (2100, 4, 0, 5, 0, False),    # Y only
    (3001, 70, 40, 0, 8, True),   # wide: beta gradient in its own kernel, 4 gamma/alpha slots per thread
    (1037, 128, 120, 1, 1, False),  # widest shape of that kernel (p, K up to 128)
]


@pytest.mark.parametrize("shape", EDGE_SHAPES, ids=lambda s: "N{}_K{}_p{}_d{}_f{}".format(*s[:5]))
@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_edge_shapes(MNL, shape, prec):
    N, K, p, d, f, icpt = shape
    prob = datagen.make_problem(N, K, p, d, f, 100 + N, intercept=icpt, theta_sd=0.3)
    th = np.random.default_rng(1).normal(0, 0.1, prob.n_theta)
    check_lgH(MNL, prob, prec, th)


@pytest.mark.parametrize("prec", PRECS)
def test_fit_matches_oracle_fit(MNL, prec):
    prob = s1(seed=12)
    th_ref, st = oracle.fit(prob)
    assert st["stop"] in ("gtol", "steptol")
    assert np.abs(oracle.loglik_grad(prob, th_ref)[1]).max() < 1e-7
    with MNL(**dev(prob), precision=prec) as m:
        th, info = m.fit()
        assert info["status"] == 0, info
        th = th.cpu().numpy()
    err = np.abs(th - th_ref).max() / np.abs(th_ref).max()
    assert err <= THETA_TOL, (prec, err, info)


def read_golden(name):
    path = os.path.join(GOLDEN, f"oracle_fit_{name}.txt")
    meta, theta = {}, []
    with open(path) as fh:
        lines = [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]
    i = lines.index("theta")
    for ln in lines[:i]:
        k, v = ln.split(None, 1)
        meta[k] = v
    theta = np.array([float(v) for v in lines[i + 1:]])
    assert theta.size == int(meta["n_theta"])
    return meta, theta


def fingerprint(prob):
    import hashlib
    h = hashlib.sha256()
    for a in (prob.X, prob.Y, prob.Z, prob.choice):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("prec", PRECS)
def test_workload1_fit_to_gradient_tolerance(MNL, prec):
    prob = datagen.config1()
    meta, th_ref = read_golden("c1")
    assert fingerprint(prob) == meta["fingerprint"]
    with MNL(**dev(prob), precision=prec) as m:
        kw = dict(gtol=1e-8) if prec == "fp64" else {}
        th, info = m.fit(**kw)
        th = th.cpu().numpy()
    assert info["status"] == 0
    if prec == "fp64":
        assert info["stop_reason"] == 1 and info["grad_inf"] < 1e-8
    assert np.abs(th - th_ref).max() / np.abs(th_ref).max() <= THETA_TOL


# ---------------------------------------------------------------------------
# Full-size workload 2 (N=200000, K=50, p=50, d=5, f=5; 2700 coefficients)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2():
    prob = datagen.config2()
    meta, th_ref = read_golden("c2")
    assert fingerprint(prob) == meta["fingerprint"], "regenerated inputs differ from the stored oracle fit"
    return prob, th_ref


def frobenius_estimate(F_gpu, entries_ref, rows, cols, n):
    """Stratified estimate of ||F_gpu - F||_F / ||F||_F from sampled oracle entries."""
    diag = rows == cols
    e2 = (F_gpu[rows, cols] - entries_ref) ** 2
    f2 = entries_ref ** 2
    nd, no = max(diag.sum(), 1), max((~diag).sum(), 1)
    num = n / nd * e2[diag].sum() + n * (n - 1) / no * e2[~diag].sum()
    den = n / nd * f2[diag].sum() + n * (n - 1) / no * f2[~diag].sum()
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("prec", PRECS)
def test_workload2_full_size(MNL, c2, prec):
    prob, th_ref = c2
    n = prob.n_theta
    l_ref, g_ref = oracle.loglik_grad(prob)
    rng = np.random.default_rng(2)
    d_idx = rng.choice(n, 60, replace=False)
    r = rng.integers(0, n, 90)
    c = rng.integers(0, n, 90)
    lo = np.concatenate([np.minimum(r, c), rng.integers(n - prob.f, n, 10)])
    hi = np.concatenate([np.maximum(r, c), rng.integers(0, n, 10)])
    rows = np.concatenate([d_idx, hi])
    cols = np.concatenate([d_idx, lo])
    F_ref = oracle.neg_hessian_entries(prob, np.zeros(n), rows, cols)
    with MNL(**dev(prob), precision=prec) as m:
        l, g = m.loglik_grad()
        g = g.cpu().numpy()
        assert abs(l - l_ref) <= TOL[prec]["l"] * abs(l_ref)
        assert rel(g, g_ref) <= TOL[prec]["g"], rel(g, g_ref)
        H = m.hessian().cpu().numpy()
        est = frobenius_estimate(-H, F_ref, rows, cols, n)
        assert est <= TOL[prec]["H"], (prec, est)
        if prec == "fp64":
            np.testing.assert_allclose(-H[rows, cols], F_ref, rtol=1e-9, atol=1e-9 * np.abs(F_ref).max())
        del H
        th, info = m.fit()
        assert info["status"] == 0, info
        th = th.cpu().numpy()
    err = np.abs(th - th_ref).max() / np.abs(th_ref).max()
    assert err <= THETA_TOL, (prec, err, info)


# ---------------------------------------------------------------------------
# Boundary behaviour
# ---------------------------------------------------------------------------

def test_host_upload_matches_device_data(MNL):
    prob = s1()
    with MNL(**dev(prob), precision="bf16") as a:
        la, ga = a.loglik_grad()
        Ha = a.hessian()
    b = MNL.with_host_upload(prob.N, prob.K, prob.p, prob.d, prob.f, precision="bf16")
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()  # noqa: E731
    b.upload(pin(prob.X), pin(prob.Y), pin(prob.Z), pin(prob.choice))
    lb, gb = b.loglik_grad()
    Hb = b.hessian()
    b.close()
    assert la == lb and torch.equal(ga, gb) and torch.equal(Ha, Hb)


def test_results_are_deterministic(MNL):
    prob = s1()
    outs = []
    for _ in range(2):
        with MNL(**dev(prob), precision="bf16") as m:
            th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
            m.newton_step(th)
            outs.append(th.cpu())
    assert torch.equal(outs[0], outs[1])


def test_invalid_choice_is_rejected(MNL):
    from paper_1404_3177_gb300._native import MnlError, MNL_ERR_INVALID_ARG
    prob = datagen.make_problem(100, 4, 2, 0, 0, 3)
    prob.choice[17] = 4
    with pytest.raises(MnlError) as e:
        MNL(**dev(prob), precision="fp64")
    assert e.value.status == MNL_ERR_INVALID_ARG


def test_nonfinite_data_is_rejected(MNL):
    from paper_1404_3177_gb300._native import MnlError, MNL_ERR_NONFINITE
    prob = datagen.make_problem(100, 4, 2, 1, 1, 3)
    prob.Z[5, 2, 0] = np.nan
    with pytest.raises(MnlError) as e:
        MNL(**dev(prob), precision="bf16")
    assert e.value.status == MNL_ERR_NONFINITE


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_unidentified_coefficient_reports_not_pd(MNL, prec):
    from paper_1404_3177_gb300._native import MnlError, MNL_ERR_NOT_PD
    prob = datagen.make_problem(500, 4, 3, 0, 0, 3)
    prob.X[:, 2] = 0.0  # a column of zeros: its coefficients do not enter l
    with MNL(**dev(prob), precision=prec) as m:
        th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
        with pytest.raises(MnlError) as e:
            m.newton_step(th)
        assert e.value.status == MNL_ERR_NOT_PD
        assert float(th.abs().max()) == 0.0  # theta untouched on error


def test_unsupported_requests(MNL):
    from paper_1404_3177_gb300 import _native as nat
    with pytest.raises(nat.MnlError) as e:
        nat.mnl_create(nat.mnl_dims(10, 300, 2, 0, 0, 0), None, nat.MNL_BF16, 0)
    assert e.value.status == nat.MNL_ERR_UNSUPPORTED
    with pytest.raises(nat.MnlError) as e:  # gamma_base = 1 needs Y columns (a gamma_0 to estimate)
        nat.mnl_create(nat.mnl_dims(10, 4, 2, 0, 1, 1), None, nat.MNL_BF16, 0)
    assert e.value.status == nat.MNL_ERR_INVALID_ARG
    with pytest.raises(nat.MnlError) as e:  # the batched calls keep gamma_0 = 0
        nat.mnl_batch_create([nat.mnl_dims(10, 4, 2, 1, 0, 1)], [nat.mnl_data(16, 16, None, 16)], nat.MNL_BF16, 0)
    assert e.value.status == nat.MNL_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# Newton solve: float64 Cholesky vs float32 factor + float64 refinement
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_mixed_and_fp64_solves_agree(MNL, prec):
    prob = s1()
    steps = {}
    for solve in ("fp64", "mixed"):
        with MNL(**dev(prob), precision=prec, solve=solve) as m:
            th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
            info = m.newton_step(th)
            steps[solve] = (th.cpu().numpy(), info)
    a, ia = steps["fp64"]
    b, ib = steps["mixed"]
    assert ia["solve_mode"] == 1 and ib["solve_mode"] == 2 and ib["fallback"] == 0 and ib["refine_steps"] >= 1
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max(), np.abs(a - b).max() / np.abs(a).max()


def test_mixed_solve_falls_back_to_fp64_on_ill_conditioned_design(MNL):
    prob = datagen.make_problem(3000, 3, 3, 0, 0, 9, theta_sd=0.3)
    rng = np.random.default_rng(4)
    prob.X[:, 2] = (prob.X[:, 1] + 1e-5 * rng.standard_normal(prob.N)).astype(np.float32)  # cond(-H) ~ 1e10
    out = {}
    for solve in ("fp64", "mixed"):
        with MNL(**dev(prob), precision="fp64", solve=solve) as m:
            th = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda")
            info = m.newton_step(th)
            out[solve] = (th.cpu().numpy(), info)
    assert out["mixed"][1]["fallback"] == 1
    assert np.array_equal(out["fp64"][0], out["mixed"][0])


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_float32_gradient_modes_stop_at_the_noise_floor(MNL, prec):
    """Few observations per coefficient: the step stops shrinking near the float32
    gradient's noise floor; the fit stops there, within the coefficient bar."""
    prob = datagen.make_problem(6000, 30, 50, 0, 0, 4242, intercept=True, theta_sd=0.3 / math.sqrt(50))
    ref, _ = oracle.fit(prob)
    with MNL(**dev(prob), precision=prec) as m:
        th, info = m.fit()
    assert info["status"] == 0 and info["stop_reason"] in (3, 5), info
    assert np.abs(th.cpu().numpy() - ref).max() / np.abs(ref).max() <= THETA_TOL


# ---------------------------------------------------------------------------
# Step halving (Sec. 3.1): a start where the full Newton step lowers l
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_step_halving_from_a_distant_start(MNL, prec):
    prob = datagen.make_problem(4000, 4, 3, 1, 2, 11, theta_sd=0.5)
    th0 = 2.0 * np.random.default_rng(7).standard_normal(prob.n_theta)
    ref, st = oracle.fit(prob, th0, maxiter=1, gtol=0.0)
    assert st["ls_evals"] == 3  # the oracle rejects t = 1 and t = 1/2 (l drops by thousands) and takes t = 1/4
    with MNL(**dev(prob), precision=prec, solve="fp64" if prec == "fp64" else "auto") as m:
        th = torch.from_numpy(th0.copy()).cuda()
        info = m.newton_step(th)
        th = th.cpu().numpy()
    assert info["halvings"] == 2 and info["ls_evals"] == 3 and info["step_scale"] == 0.25, info
    assert oracle.loglik_grad(prob, th)[0] > oracle.loglik_grad(prob, th0)[0]
    tol = 1e-9 if prec == "fp64" else 5e-2  # relative to the step; BF16: the Hessian's 2e-3 error
    assert np.abs(th - ref).max() <= tol * np.abs(ref - th0).max()
