"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: values the
paper prints, closed forms, brute force of the paper's own formulas written
independently here, textbook algorithms, and exact invariances.  A dropped
term, a wrong sign, a wrong index or a transposed operand anywhere in the
oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_kv(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()[:2]
            out[k] = v
    return out


def small(N=60, K=4, p=3, d=2, f=2, seed=7, gamma_base=0, intercept=True, theta_sd=0.4):
    return datagen.make_problem(N, K, p, d, f, seed, gamma_base=gamma_base, intercept=intercept, theta_sd=theta_sd)


def rand_theta(prob, seed=3, sd=0.3):
    return np.random.default_rng(seed).normal(0, sd, prob.n_theta)


# ---------------------------------------------------------------------------
# Independent restatements of the paper's formulas (pure Python loops).
# ---------------------------------------------------------------------------

def split_theta(prob, theta):
    """beta[K][p] (beta_0 = 0), gamma[K][d] (gamma_0 = 0 unless estimated), alpha[f] per eq. "theta vec"."""
    K, p, d = prob.K, prob.p, prob.d
    nb = (K - 1) * p
    beta = np.zeros((K, p))
    beta[1:] = theta[:nb].reshape(K - 1, p)
    gamma = np.zeros((K, d))
    if prob.gamma_base:
        gamma[:] = theta[nb:nb + K * d].reshape(K, d)
        alpha = theta[nb + K * d:]
    else:
        gamma[1:] = theta[nb:nb + (K - 1) * d].reshape(K - 1, d)
        alpha = theta[nb + (K - 1) * d:]
    return beta, gamma, alpha


def paper_V(prob, theta, i):
    """Normalized utilities V_i1..V_i,K-1 (eq. "normalized utility"; Z_ik means Z_ik - Z_i0)."""
    beta, gamma, alpha = split_theta(prob, theta)
    X = prob.X.astype(np.float64)
    Y = prob.Y.astype(np.float64)
    Z = prob.Z.astype(np.float64)
    V = []
    for k in range(1, prob.K):
        v = 0.0
        for j in range(prob.p):
            v += X[i, j] * beta[k, j]
        for j in range(prob.d):
            v += Y[i, k, j] * gamma[k, j] - Y[i, 0, j] * gamma[0, j]
        for j in range(prob.f):
            v += (Z[i, k, j] - Z[i, 0, j]) * alpha[j]
        V.append(v)
    return V


def paper_loglik_and_probs(prob, theta):
    """eqs. "base probability", "probability" and "log-lik function" literally (no max shift)."""
    l = 0.0
    P = np.zeros((prob.N, prob.K))
    for i in range(prob.N):
        V = paper_V(prob, theta, i)
        s = 1.0 + sum(math.exp(v) for v in V)
        P[i, 0] = 1.0 / s
        for k in range(1, prob.K):
            P[i, k] = P[i, 0] * math.exp(V[k - 1])
        l += -math.log(s) + sum(V[k - 1] for k in range(1, prob.K) if prob.choice[i] == k)
    return l, P


# ---------------------------------------------------------------------------
# Parameter counts printed in the paper
# ---------------------------------------------------------------------------

def test_param_counts_printed_in_paper():
    with open(os.path.join(GOLDEN, "param_counts.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for r in rows:
        K, p, d, f, gb, count = map(int, r[1:7])
        assert oracle.num_params(K, p, d, f, gb) == count, r


def test_param_counts_of_the_workloads():
    # (K-1)(p+d)+f with gamma_0 not estimated: 22, 2700, 9910
    assert oracle.num_params(5, 4, 1, 2, 0) == 22
    assert oracle.num_params(50, 50, 5, 5, 0) == 2700
    assert oracle.num_params(100, 100, 0, 10, 0) == 9910


# ---------------------------------------------------------------------------
# Log-likelihood
# ---------------------------------------------------------------------------

def test_loglik_at_zero_matches_appendix_c_printed_value():
    g = _read_kv("appc_nnet_initial_value.txt")
    N, K = int(g["N"]), int(g["K"])
    # problem X of App. C: individual-specific data only, no intercept
    prob = datagen.make_problem(N, K, 50, 0, 0, 11, intercept=False)
    l0 = oracle.loglik(prob, np.zeros(prob.n_theta))
    assert abs(-l0 - float(g["neg_loglik_at_zero"])) <= 0.5 * 10 ** -int(g["printed_decimals"])


@pytest.mark.parametrize("shape", [(50, 3, 2, 1, 1), (40, 6, 1, 0, 3), (30, 2, 3, 2, 0)])
def test_loglik_at_zero_closed_form(shape):
    N, K, p, d, f = shape
    prob = datagen.make_problem(N, K, p, d, f, 5)
    assert oracle.loglik(prob) == pytest.approx(-N * math.log(K), rel=1e-14)


@pytest.mark.parametrize("gamma_base", [0, 1])
def test_loglik_and_probs_match_paper_formulas_brute_force(gamma_base):
    prob = small(gamma_base=gamma_base)
    th = rand_theta(prob)
    l_ref, P_ref = paper_loglik_and_probs(prob, th)
    P, l = oracle.probs(prob, th)
    assert l == pytest.approx(l_ref, rel=1e-13)
    np.testing.assert_allclose(P, P_ref, rtol=1e-12, atol=1e-15)
    assert oracle.loglik_grad(prob, th)[0] == pytest.approx(l_ref, rel=1e-13)


def test_loglik_is_stable_for_large_utilities():
    prob = small()
    th = rand_theta(prob, sd=80.0)  # exp would overflow without a max shift
    l, g = oracle.loglik_grad(prob, th)
    assert np.isfinite(l) and np.all(np.isfinite(g)) and l <= 0


# ---------------------------------------------------------------------------
# Gradient and Hessian: finite differences, symmetry, concavity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gamma_base", [0, 1])
def test_gradient_matches_central_differences(gamma_base):
    prob = small(gamma_base=gamma_base)
    th = rand_theta(prob)
    _, g = oracle.loglik_grad(prob, th)
    fd = np.empty_like(g)
    for j in range(prob.n_theta):
        h = 1e-5 * max(1.0, abs(th[j]))
        e = np.zeros_like(th)
        e[j] = h
        fd[j] = (oracle.loglik(prob, th + e) - oracle.loglik(prob, th - e)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-7 * np.abs(g).max())


@pytest.mark.parametrize("gamma_base", [0, 1])
def test_hessian_matches_central_differences_of_gradient(gamma_base):
    prob = small(gamma_base=gamma_base)
    th = rand_theta(prob)
    F = oracle.neg_hessian(prob, th)
    fd = np.empty_like(F)
    for j in range(prob.n_theta):
        h = 1e-5 * max(1.0, abs(th[j]))
        e = np.zeros_like(th)
        e[j] = h
        fd[:, j] = -(oracle.loglik_grad(prob, th + e)[1] - oracle.loglik_grad(prob, th - e)[1]) / (2 * h)
    np.testing.assert_allclose(F, fd, rtol=1e-6, atol=1e-6 * np.abs(F).max())


def test_hessian_symmetric_and_negative_definite():
    prob = small(N=200, K=5, p=3, d=2, f=2)
    F = oracle.neg_hessian(prob, rand_theta(prob))
    assert np.array_equal(F, F.T)
    assert np.linalg.eigvalsh(F).min() > 0
    assert oracle.cholesky(F) is not None


def test_hessian_thread_count_does_not_change_bits():
    prob = small(N=300, K=6, p=4, d=2, f=3)
    th = rand_theta(prob)
    assert np.array_equal(oracle.neg_hessian(prob, th, nthreads=1), oracle.neg_hessian(prob, th, nthreads=4))


def test_hessian_equals_dense_irls_form_for_x_only_model():
    """Eq. "old Hessian formula": H = -Xt^T Wt Xt with block-diagonal Xt and W_kt = diag(P_k (delta_kt - P_t))."""
    prob = small(N=40, K=4, p=3, d=0, f=0)
    th = rand_theta(prob)
    _, P = paper_loglik_and_probs(prob, th)
    N, K, p = prob.N, prob.K, prob.p
    X = prob.X.astype(np.float64)
    Xt = np.zeros(((K - 1) * N, (K - 1) * p))
    for k in range(K - 1):
        Xt[k * N:(k + 1) * N, k * p:(k + 1) * p] = X
    Wt = np.zeros(((K - 1) * N, (K - 1) * N))
    for k in range(1, K):
        for t in range(1, K):
            w = P[:, k] * ((1.0 if k == t else 0.0) - P[:, t])
            Wt[(k - 1) * N:k * N, (t - 1) * N:t * N] = np.diag(w)
    H_irls = -Xt.T @ Wt @ Xt
    np.testing.assert_allclose(-oracle.neg_hessian(prob, th), H_irls, rtol=1e-12, atol=1e-12)
    # gradient Xt^T (y - P), y stacked per alternative k = 1..K-1
    yv = np.concatenate([(prob.choice == k).astype(np.float64) for k in range(1, K)])
    Pv = np.concatenate([P[:, k] for k in range(1, K)])
    np.testing.assert_allclose(oracle.loglik_grad(prob, th)[1], Xt.T @ (yv - Pv), rtol=1e-12, atol=1e-12)


def test_hessian_blocks_match_block_formula_with_generic_coefficients():
    """Eq. "hessian block": H_nm = -M_n^T W_nm M_m; H_{n,alpha} = -sum_k M_n^T W_nk Z_k;
    H_{alpha,alpha} = -sum_{k,t} Z_k^T W_kt Z_t, with Z_k = Z_k - Z_0 (normalization) and W_nm as above."""
    prob = small(N=50, K=4, p=2, d=2, f=2)
    th = rand_theta(prob)
    _, P = paper_loglik_and_probs(prob, th)
    K, p, d, f = prob.K, prob.p, prob.d, prob.f
    X = prob.X.astype(np.float64)
    Y = prob.Y.astype(np.float64)
    Zn = prob.Z.astype(np.float64) - prob.Z[:, :1, :].astype(np.float64)

    def W(n, m):
        return P[:, n] * ((1.0 if n == m else 0.0) - P[:, m])

    # coefficient chunks: beta_k -> M = X, gamma_k -> M = Y_k (k = 1..K-1)
    chunks = [("b", k) for k in range(1, K)] + [("g", k) for k in range(1, K)]

    def M(ch):
        typ, k = ch
        return X if typ == "b" else Y[:, k, :]

    H = np.zeros((prob.n_theta, prob.n_theta))
    offs, o = {}, 0
    for ch in chunks:
        offs[ch] = o
        o += p if ch[0] == "b" else d
    oa = o
    for a in chunks:
        for b in chunks:
            blk = -M(a).T @ (W(a[1], b[1])[:, None] * M(b))
            H[offs[a]:offs[a] + M(a).shape[1], offs[b]:offs[b] + M(b).shape[1]] = blk
        cross = -sum(M(a).T @ (W(a[1], k)[:, None] * Zn[:, k, :]) for k in range(1, K))
        H[offs[a]:offs[a] + M(a).shape[1], oa:] = cross
        H[oa:, offs[a]:offs[a] + M(a).shape[1]] = cross.T
    H[oa:, oa:] = -sum(Zn[:, k, :].T @ (W(k, t)[:, None] * Zn[:, t, :]) for k in range(1, K) for t in range(1, K))
    np.testing.assert_allclose(-oracle.neg_hessian(prob, th), H, rtol=1e-12, atol=1e-12)


def test_z_normalization_shift_invariance():
    """Only Z_ik - Z_i0 enters (Sec. 2.1): adding a per-observation constant to every alternative's Z changes nothing."""
    prob = small(N=80, K=5, p=2, d=1, f=3)
    prob.Z = (np.round(prob.Z * 256) / 256).astype(np.float32)  # 8 fractional bits: the shift below is exact
    th = rand_theta(prob)
    l0, g0 = oracle.loglik_grad(prob, th)
    F0 = oracle.neg_hessian(prob, th)
    shift = np.random.default_rng(1).integers(-8, 9, size=(prob.N, 1, prob.f)).astype(np.float32)
    prob.Z = (prob.Z + shift).astype(np.float32)
    l1, g1 = oracle.loglik_grad(prob, th)
    assert l1 == l0 and np.array_equal(g1, g0) and np.array_equal(oracle.neg_hessian(prob, th), F0)


def test_hessian_entries_sampler_matches_full_matrix():
    for gb in (0, 1):
        prob = small(N=70, K=5, p=3, d=2, f=2, gamma_base=gb)
        th = rand_theta(prob)
        F = oracle.neg_hessian(prob, th)
        rng = np.random.default_rng(0)
        r = rng.integers(0, prob.n_theta, 60)
        c = rng.integers(0, prob.n_theta, 60)
        np.testing.assert_allclose(oracle.neg_hessian_entries(prob, th, r, c), F[r, c], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Special cases that reduce to textbook results
# ---------------------------------------------------------------------------

def test_two_alternatives_reduce_to_binary_logistic_regression():
    """K = 2 is binary logistic regression (Sec. 2.1): g = X^T (y - s), -H = X^T diag(s(1-s)) X,
    and the fitted coefficients equal a textbook IRLS fit."""
    prob = datagen.make_problem(400, 2, 3, 0, 0, 21, intercept=True, theta_sd=0.8)
    X = prob.X.astype(np.float64)
    y = (prob.choice == 1).astype(np.float64)
    th = rand_theta(prob)
    s = 1.0 / (1.0 + np.exp(-(X @ th)))
    l, g = oracle.loglik_grad(prob, th)
    assert l == pytest.approx(np.sum(y * np.log(s) + (1 - y) * np.log(1 - s)), rel=1e-13)
    np.testing.assert_allclose(g, X.T @ (y - s), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.neg_hessian(prob, th), X.T @ ((s * (1 - s))[:, None] * X), rtol=1e-12)
    # textbook IRLS: beta <- (X^T W X)^{-1} X^T W z, z = X beta + (y - s)/w
    b = np.zeros(3)
    for _ in range(50):
        s = 1.0 / (1.0 + np.exp(-(X @ b)))
        w = s * (1 - s)
        zz = X @ b + (y - s) / w
        b = np.linalg.solve(X.T @ (w[:, None] * X), X.T @ (w * zz))
    th_hat, st = oracle.fit(prob)
    np.testing.assert_allclose(th_hat, b, rtol=1e-10, atol=1e-12)
    assert st["stop"] == "gtol"


def test_intercept_only_mle_is_log_frequency_ratio():
    """With only the intercept (X = 1), the MLE of xi_k - xi_0 is ln(n_k / n_0)."""
    prob = datagen.make_problem(3000, 5, 1, 0, 0, 31, intercept=True, theta_sd=0.7)
    th_hat, st = oracle.fit(prob)
    n = np.bincount(prob.choice, minlength=5).astype(np.float64)
    np.testing.assert_allclose(th_hat, np.log(n[1:] / n[0]), rtol=1e-10, atol=1e-12)
    assert st["stop"] == "gtol"


def test_saturated_one_hot_design_gives_group_log_ratios():
    """X = one-hot group indicator (no intercept): beta_k[g] = ln(n_gk / n_g0) for every group g."""
    G, K, N = 3, 4, 2400
    prob = datagen.make_problem(N, K, G, 0, 0, 41, intercept=False)
    grp = np.arange(N) % G
    prob.X = np.eye(G, dtype=np.float32)[grp]
    rng = np.random.default_rng(2)
    prob.choice = rng.integers(0, K, N).astype(np.int32)
    th_hat, _ = oracle.fit(prob)
    beta = th_hat.reshape(K - 1, G)
    for g in range(G):
        n = np.bincount(prob.choice[grp == g], minlength=K).astype(np.float64)
        np.testing.assert_allclose(beta[:, g], np.log(n[1:] / n[0]), rtol=1e-10, atol=1e-12)


def test_cholesky_and_solve_match_library_routines():
    rng = np.random.default_rng(4)
    B = rng.normal(size=(37, 37))
    A = B @ B.T + 37 * np.eye(37)
    L = oracle.cholesky(A)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    b = rng.normal(size=37)
    np.testing.assert_allclose(oracle.cholesky_solve(L, b), np.linalg.solve(A, b), rtol=1e-10)
    A[5, 5] = -1.0
    assert oracle.cholesky(A) is None


# ---------------------------------------------------------------------------
# Newton-Raphson
# ---------------------------------------------------------------------------

def test_newton_fit_reaches_stationary_point_of_workload_1():
    prob = datagen.config1()
    th_hat, st = oracle.fit(prob, gtol=1e-8)
    assert st["stop"] == "gtol" and st["grad_inf"] < 1e-8
    l, g = oracle.loglik_grad(prob, th_hat)
    assert np.abs(g).max() < 1e-8
    assert l > oracle.loglik(prob)
    # statistical sanity: the estimate is within a few standard errors of the truth
    se = np.sqrt(np.diag(np.linalg.inv(oracle.neg_hessian(prob, th_hat))))
    assert np.all(np.abs(th_hat - prob.theta_true) < 5 * se)


def test_line_search_halves_until_loglik_not_lower():
    """A start far from the optimum forces step halving; every accepted step raises l (Sec. 3.1)."""
    prob = small(N=200, K=4, p=2, d=1, f=1)
    th0 = rand_theta(prob, sd=6.0)
    th1, st1 = oracle.fit(prob, th0, maxiter=1, gtol=0.0)
    assert oracle.loglik(prob, th1) >= oracle.loglik(prob, th0)
    th_hat, st = oracle.fit(prob, th0, gtol=1e-9)
    assert st["stop"] in ("gtol", "steptol") and st["ls_evals"] > st["iters"]  # some steps were halved
    assert np.abs(oracle.loglik_grad(prob, th_hat)[1]).max() < 1e-8


def test_singular_design_reports_not_positive_definite():
    """A duplicated X column makes -H singular (App. B condition 1): the Cholesky must fail."""
    prob = small(N=100, K=3, p=3, d=0, f=0)
    prob.X[:, 2] = prob.X[:, 1]
    F = oracle.neg_hessian(prob, rand_theta(prob))
    assert oracle.cholesky(F) is None or np.linalg.eigvalsh(F).min() < 1e-8 * np.abs(F).max()


# ---------------------------------------------------------------------------
# Standard errors (the package's summary table): sqrt(diag((-H)^-1)) at the estimate
# ---------------------------------------------------------------------------

def test_std_errors_intercept_only_closed_form():
    """Intercept only: Var(ln(n_k / n_0)) = 1/n_k + 1/n_0 (multinomial log-odds)."""
    prob = datagen.make_problem(3000, 5, 1, 0, 0, 31, intercept=True, theta_sd=0.7)
    th_hat, _ = oracle.fit(prob)
    n = np.bincount(prob.choice, minlength=5).astype(np.float64)
    np.testing.assert_allclose(oracle.std_errors(prob, th_hat), np.sqrt(1.0 / n[1:] + 1.0 / n[0]), rtol=1e-9)


def test_std_errors_saturated_groups_closed_form():
    """One-hot groups: Var(beta_k[g]) = 1/n_gk + 1/n_g0, independently per group."""
    G, K, N = 3, 4, 2400
    prob = datagen.make_problem(N, K, G, 0, 0, 41, intercept=False)
    grp = np.arange(N) % G
    prob.X = np.eye(G, dtype=np.float32)[grp]
    prob.choice = np.random.default_rng(2).integers(0, K, N).astype(np.int32)
    th_hat, _ = oracle.fit(prob)
    se = oracle.std_errors(prob, th_hat).reshape(K - 1, G)
    for g in range(G):
        n = np.bincount(prob.choice[grp == g], minlength=K).astype(np.float64)
        np.testing.assert_allclose(se[:, g], np.sqrt(1.0 / n[1:] + 1.0 / n[0]), rtol=1e-9)


def test_std_errors_binary_logit_textbook():
    """K = 2: sqrt(diag((X^T W X)^-1)) with W = p(1 - p) at the estimate, formed here with NumPy."""
    prob = datagen.make_problem(400, 2, 3, 0, 0, 21, intercept=True, theta_sd=0.8)
    th_hat, _ = oracle.fit(prob)
    X = prob.X.astype(np.float64)
    pr = 1.0 / (1.0 + np.exp(-(X @ th_hat)))
    info = X.T @ (X * (pr * (1.0 - pr))[:, None])
    np.testing.assert_allclose(oracle.std_errors(prob, th_hat), np.sqrt(np.diag(np.linalg.inv(info))), rtol=1e-9)
