"""Pins of the oracle's observation weights (case weights: the package's
`weights` argument, Sec. 2.3; the paper does not define them further, so the
reading is that observation i counts w_i times).  Each pin is fixed by that
reading, not by the oracle's own code:
  * unit weights change nothing (bit for bit);
  * integer weights equal repeating the rows (l, g, -H, and the fit);
  * zero weights equal dropping the rows;
  * scaling all weights by c scales l, g and -H by c;
  * the weighted gradient is the central difference of the weighted l;
  * K = 2 is weighted binary logistic regression: -H = X^T diag(w s (1 - s)) X
    and the fit equals a textbook weighted IRLS written here with NumPy.
"""
import numpy as np

import oracle
from paper_1404_3177_gb300 import datagen


def weighted(prob, w):
    prob.w = np.ascontiguousarray(w, dtype=np.float32)
    return prob


def rows(prob, idx):
    return datagen.Problem(len(idx), prob.K, prob.p, prob.d, prob.f, prob.gamma_base, prob.X[idx], prob.Y[idx],
                           prob.Z[idx], prob.choice[idx], prob.theta_true)


def base(seed=3, N=300):
    return datagen.make_problem(N, 4, 3, 1, 2, seed, theta_sd=0.4)


def test_unit_weights_change_nothing():
    p0 = base()
    th = np.random.default_rng(1).normal(0, 0.2, p0.n_theta)
    l0, g0 = oracle.loglik_grad(p0, th)
    F0 = oracle.neg_hessian(p0, th)
    p1 = weighted(base(), np.ones(p0.N))
    l1, g1 = oracle.loglik_grad(p1, th)
    assert l1 == l0 and np.array_equal(g1, g0)
    assert np.array_equal(oracle.neg_hessian(p1, th), F0)


def test_integer_weights_equal_repeated_rows():
    p = base()
    w = np.random.default_rng(2).integers(0, 4, p.N)
    th = np.random.default_rng(3).normal(0, 0.2, p.n_theta)
    pw = weighted(base(), w)
    pr = rows(base(), np.repeat(np.arange(p.N), w))
    lw, gw = oracle.loglik_grad(pw, th)
    lr, gr = oracle.loglik_grad(pr, th)
    assert abs(lw - lr) <= 1e-12 * abs(lr)
    assert np.abs(gw - gr).max() <= 1e-12 * np.abs(gr).max()
    Fw, Fr = oracle.neg_hessian(pw, th), oracle.neg_hessian(pr, th)
    assert np.abs(Fw - Fr).max() <= 1e-12 * np.abs(Fr).max()
    tw, _ = oracle.fit(pw)
    tr, _ = oracle.fit(pr)
    assert np.abs(tw - tr).max() <= 1e-9 * np.abs(tr).max()


def test_zero_weights_drop_rows():
    p = base(N=400)
    keep = np.arange(p.N) % 3 != 0
    th = np.random.default_rng(4).normal(0, 0.2, p.n_theta)
    lw, gw = oracle.loglik_grad(weighted(base(N=400), keep.astype(np.float32)), th)
    ld, gd = oracle.loglik_grad(rows(base(N=400), np.flatnonzero(keep)), th)
    assert abs(lw - ld) <= 1e-13 * abs(ld)
    assert np.abs(gw - gd).max() <= 1e-13 * np.abs(gd).max()


def test_scaled_weights_scale_everything():
    p = base()
    w = np.random.default_rng(5).uniform(0.1, 2.0, p.N).astype(np.float32)
    th = np.random.default_rng(6).normal(0, 0.2, p.n_theta)
    l1, g1 = oracle.loglik_grad(weighted(base(), w), th)
    l2, g2 = oracle.loglik_grad(weighted(base(), 4 * w), th)  # exact in float32 (power of two)
    assert abs(l2 - 4 * l1) <= 1e-13 * abs(l2)
    assert np.abs(g2 - 4 * g1).max() <= 1e-13 * np.abs(g2).max()
    F1, F2 = oracle.neg_hessian(weighted(base(), w), th), oracle.neg_hessian(weighted(base(), 4 * w), th)
    assert np.abs(F2 - 4 * F1).max() <= 1e-13 * np.abs(F2).max()


def test_weighted_gradient_is_the_derivative_of_the_weighted_loglik():
    p = weighted(base(), np.random.default_rng(7).uniform(0.0, 3.0, 300))
    th = np.random.default_rng(8).normal(0, 0.3, p.n_theta)
    _, g = oracle.loglik_grad(p, th)
    for j in range(p.n_theta):
        h = 1e-5 * max(1.0, abs(th[j]))
        e = np.zeros(p.n_theta)
        e[j] = h
        fd = (oracle.loglik(p, th + e) - oracle.loglik(p, th - e)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j]))


def test_k2_weighted_is_weighted_logistic_regression():
    p = datagen.make_problem(2000, 2, 3, 0, 0, 9, theta_sd=0.7)
    w = np.random.default_rng(10).uniform(0.2, 3.0, p.N).astype(np.float32)
    pw = weighted(p, w)
    X = p.X.astype(np.float64)
    y = (p.choice == 1).astype(np.float64)
    wd = w.astype(np.float64)
    beta = np.zeros(3)
    for _ in range(50):  # textbook weighted IRLS
        s = 1 / (1 + np.exp(-X @ beta))
        Hm = X.T @ (X * (wd * s * (1 - s))[:, None])
        step = np.linalg.solve(Hm, X.T @ (wd * (y - s)))
        beta += step
        if np.abs(step).max() < 1e-14:
            break
    s = 1 / (1 + np.exp(-X @ beta))
    F = oracle.neg_hessian(pw, beta)
    assert np.abs(F - X.T @ (X * (wd * s * (1 - s))[:, None])).max() <= 1e-10 * np.abs(F).max()
    th, _ = oracle.fit(pw)
    assert np.abs(th - beta).max() <= 1e-9 * np.abs(beta).max()


def test_negative_or_nonfinite_weights_are_rejected():
    assert oracle.check(weighted(base(), -np.ones(300))) != 0
    w = np.ones(300)
    w[7] = np.nan
    assert oracle.check(weighted(base(), w)) != 0
