"""Collinearity check and dropped columns on the GPU (Sec. 2.3 `linDepTol`;
App. B) against the oracle.

  * mnl_check_collinear: the flags (integers) equal the oracle's, bit for bit,
    on problems with planted dependencies in X, in one class's Y_k, in Y_0 (only
    counted with gamma_base = 1), in Z (a generic variable that does not vary
    over the alternatives, and a combination of the differences), on blocks
    wider than one register tile with ragged ends, on more columns than
    observations, and on full-rank data (no flags).  Every planted dependency
    is exact, so the residual norms sit many orders of magnitude away from the
    threshold and the two float64 computations (Gram-Schmidt on the data, an
    in-order Cholesky of the Gram matrix) must take the same decisions.
  * Workload-3 size (N=500000, K=100, p=100, f=10) with one planted column:
    exactly that flag, X's flags equal the oracle's on the whole X, and Z has
    none.
  * mnl_drop_columns + mnl_fit: the fit of the full (singular) model with the
    flagged columns removed equals the oracle's fit of the reduced problem
    (the data without those columns): 1e-6 relative on the kept
    coefficients, exactly zero on the dropped ones, in FP64, BF16, truncated
    Newton and with gamma_base = 1; without the drop the fit reports a
    singular -H.  Standard errors: NaN for the dropped coefficients, the
    reduced oracle's for the others.
"""
import numpy as np
import pytest

import oracle
from oracle import collinear
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

THETA_TOL = 1e-6


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300 import api as mod
    return mod


def dev(prob):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a.size else None  # noqa: E731
    return dict(X=t(prob.X), Y=t(prob.Y), Z=t(prob.Z), choice=torch.from_numpy(prob.choice).cuda(), K=prob.K,
                gamma_base=prob.gamma_base)


def planted(gamma_base=0, N=3001, seed=41):
    pr = datagen.make_problem(N, 6, 9, 2, 4, seed, theta_sd=0.3, gamma_base=gamma_base)
    pr.X[:, 3] = pr.X[:, 1] - 2 * pr.X[:, 2]
    pr.X[:, 8] = 0.5 * pr.X[:, 0]          # a multiple of the intercept
    pr.Y[:, 2, 1] = 3 * pr.Y[:, 2, 0]       # one class's Y block
    pr.Y[:, 0, 1] = -pr.Y[:, 0, 0]          # Y_0: counts only when gamma_0 is estimated
    pr.Z[:, :, 1] = pr.Z[:, :1, 1] + 0.25   # no variation over the alternatives
    pr.Z[:, :, 3] = pr.Z[:, :, 0] - pr.Z[:, :, 2]
    return pr


def wide(seed=43):
    pr = datagen.make_problem(2500, 4, 70, 0, 13, seed, theta_sd=0.2)
    pr.X[:, 33] = pr.X[:, 5] + pr.X[:, 6]
    pr.X[:, 69] = pr.X[:, :11].astype(np.float64).sum(axis=1)  # rounded to float32 once
    pr.X[:, 40] = pr.X[:, 39]
    pr.Z[:, :, 12] = 2 * pr.Z[:, :, 7]
    return pr


def short(seed=47):
    # more columns than observations: at most 50 X columns can be independent
    return datagen.make_problem(50, 3, 60, 1, 2, seed, theta_sd=0.2)


CASES = {
    "planted": lambda: planted(0),
    "planted_gamma0": lambda: planted(1),
    "wide": wide,
    "short": short,
    "full_rank": lambda: datagen.make_problem(4000, 7, 12, 3, 5, 49, theta_sd=0.3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_flags_equal_the_oracle(api, name):
    pr = CASES[name]()
    want = collinear.check(pr, 1e-6)
    for prec in ("fp64", "bf16"):
        with api.MNL(**dev(pr), precision=prec) as m:
            got = m.check_collinear(1e-6)
        assert got.tolist() == want.tolist(), (prec, np.flatnonzero(got), np.flatnonzero(want))
    if name == "planted":
        p, K, d = pr.p, pr.K, pr.d
        assert np.flatnonzero(want).tolist() == [3, 8, p + 2 * d + 1, p + K * d + 1, p + K * d + 3]
    if name == "full_rank":
        assert want.sum() == 0


def test_workload3_size_planted_column(api):
    pr = datagen.config3()
    pr.X[:, 99] = pr.X[:, 0] + pr.X[:, 1]
    with api.MNL(**dev(pr), precision="bf16") as m:
        got = m.check_collinear(1e-6)
    assert np.flatnonzero(got).tolist() == [99]
    assert got[:pr.p].tolist() == collinear.dependent_columns(pr.X, 1e-6).tolist()
    # Z: a sample of the stacked differences has full rank, so the whole block has too
    sub = datagen.Problem(20000, pr.K, pr.p, pr.d, pr.f, 0, pr.X[:20000], pr.Y[:20000], pr.Z[:20000],
                          pr.choice[:20000], pr.theta_true)
    assert collinear.dependent_columns(collinear.z_differences(sub), 1e-6).sum() == 0


def reduced(pr, flags):
    """The problem without the flagged columns (every flagged Y column must be flagged in every class used)."""
    p, K, d, f = pr.p, pr.K, pr.d, pr.f
    kx = np.flatnonzero(flags[:p] == 0)
    fy = flags[p:p + K * d].reshape(K, d)[(0 if pr.gamma_base else 1):]
    assert (fy == fy[0]).all(), "a Y column must be dropped in every class for a reduced problem"
    ky = np.flatnonzero(fy[0] == 0)
    kz = np.flatnonzero(flags[p + K * d:] == 0)
    return datagen.Problem(pr.N, K, len(kx), len(ky), len(kz), pr.gamma_base,
                           np.ascontiguousarray(pr.X[:, kx]), np.ascontiguousarray(pr.Y[:, :, ky]),
                           np.ascontiguousarray(pr.Z[:, :, kz]), pr.choice, None)


def fit_case(gamma_base):
    pr = datagen.make_problem(6007, 5, 6, 2, 3, 53, theta_sd=0.3, gamma_base=gamma_base)
    pr.X[:, 4] = pr.X[:, 1] - 2 * pr.X[:, 2]
    pr.Z[:, :, 1] = pr.Z[:, :1, 1] + 1.5
    pr.Y[:, :, 1] = 0.5 * pr.Y[:, :, 0]
    return pr


@pytest.mark.parametrize("mode", ["fp64", "bf16", "truncated", "fp64_gamma0", "bf16_gamma0"])
def test_fit_without_dropped_columns_equals_the_reduced_oracle_fit(api, mode):
    gb = 1 if mode.endswith("gamma0") else 0
    pr = fit_case(gb)
    flags = collinear.check(pr, 1e-6)
    mask = collinear.theta_mask(pr, flags)
    red = reduced(pr, flags)
    th_red, _ = oracle.fit(red)
    prec = "fp64" if mode.startswith(("fp64", "truncated")) else "bf16"
    kw = dict(precision=prec, truncated=mode == "truncated")
    with api.MNL(**dev(pr), **kw) as m:
        got = m.check_collinear(1e-6)
        assert got.tolist() == flags.tolist()
        m.drop_columns(got)
        th, info = m.fit()
        th = th.cpu().numpy()
        assert info["status"] == 0, info
        assert np.all(th[mask == 1] == 0.0)
        kept = th[mask == 0]
        assert np.abs(kept - th_red).max() <= THETA_TOL * np.abs(th_red).max(), np.abs(kept - th_red).max()
        if mode == "fp64":
            se = m.std_errors(torch.from_numpy(th).cuda()).cpu().numpy()
            assert np.all(np.isnan(se[mask == 1]))
            se_red = oracle.std_errors(red, th_red)
            assert np.abs(se[mask == 0] - se_red).max() <= 1e-8 * se_red.max()
        if prec == "fp64" and mode != "truncated":
            m.drop_columns(None)  # the full model: the Z column without variation makes -H singular
            with pytest.raises(Exception, match="not positive definite|NOT_PD|singular"):
                m.fit()
