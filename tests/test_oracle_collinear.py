"""Pins of the oracle's collinearity check (Sec. 2.3 `linDepTol`; App. B).

Each pin is fixed by linear algebra or by the paper's statement of the check,
not by the oracle's own code:
  * a random full-rank block drops nothing;
  * the later of two equal columns, a linear combination of earlier columns and
    a zero column are dropped; the earlier columns are kept;
  * the number of kept columns equals the rank from NumPy's SVD
    (`numpy.linalg.matrix_rank`) on random low-rank blocks, and the kept
    columns have full rank;
  * an intercept with a full set of group dummies (the "dummy trap") drops
    exactly the last dummy;
  * the threshold in closed form: for b = a + eps * e with e orthogonal to a
    and ||e|| = ||a||, b is dropped exactly when tol >= eps / sqrt(1 + eps^2);
  * scaling columns by powers of two changes nothing;
  * a generic variable that does not vary over the alternatives has zero
    differences Z_ik - Z_i0 and is dropped (App. B, condition 2);
  * Y_0 is checked only when gamma_0 is estimated; the coefficient mask maps
    an X column to beta_k for every k.
"""
import numpy as np
import pytest

from oracle import collinear
from paper_1404_3177_gb300 import datagen


def rand(n, c, seed):
    return np.random.default_rng(seed).normal(size=(n, c))


def test_full_rank_block_drops_nothing():
    assert collinear.dependent_columns(rand(500, 12, 1), 1e-6).sum() == 0


def test_duplicate_combination_and_zero_columns():
    A = rand(400, 6, 2)
    M = np.column_stack([A[:, 0], A[:, 1], A[:, 0], A[:, 2], 2.0 * A[:, 1] - 0.5 * A[:, 2], np.zeros(400), A[:, 3]])
    flags = collinear.dependent_columns(M, 1e-6)
    assert flags.tolist() == [0, 0, 1, 0, 1, 1, 0]


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_kept_count_equals_svd_rank(seed):
    rng = np.random.default_rng(seed)
    r, c = int(rng.integers(2, 9)), int(rng.integers(10, 16))
    M = rng.normal(size=(300, r)) @ rng.normal(size=(r, c))
    M = np.column_stack([M, rng.normal(size=(300, 2))])[:, rng.permutation(c + 2)]
    flags = collinear.dependent_columns(M, 1e-6)
    kept = np.flatnonzero(flags == 0)
    assert kept.size == np.linalg.matrix_rank(M)
    assert np.linalg.matrix_rank(M[:, kept]) == kept.size


def test_dummy_trap_drops_the_last_dummy():
    g = np.random.default_rng(6).integers(0, 4, 200)
    D = (g[:, None] == np.arange(4)[None, :]).astype(float)
    M = np.column_stack([np.ones(200), rand(200, 1, 7), D])
    assert collinear.dependent_columns(M, 1e-6).tolist() == [0, 0, 0, 0, 0, 1]


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_threshold_closed_form(eps):
    rng = np.random.default_rng(8)
    a = rng.normal(size=256)
    e = rng.normal(size=256)
    e -= a * (a @ e) / (a @ a)
    e *= np.linalg.norm(a) / np.linalg.norm(e)
    M = np.column_stack([a, a + eps * e])
    ratio = eps / np.sqrt(1 + eps * eps)
    assert collinear.dependent_columns(M, ratio * (1 - 1e-3)).tolist() == [0, 0]
    assert collinear.dependent_columns(M, ratio * (1 + 1e-3)).tolist() == [0, 1]


def test_power_of_two_scaling_changes_nothing():
    A = rand(300, 5, 9)
    M = np.column_stack([A, A[:, 1] + A[:, 3]])
    s = 2.0 ** np.array([-7, 3, 0, 11, -2, 5])
    assert collinear.dependent_columns(M * s, 1e-6).tolist() == collinear.dependent_columns(M, 1e-6).tolist()


def problem(gamma_base=0):
    return datagen.make_problem(600, 5, 4, 2, 3, 11, theta_sd=0.3, gamma_base=gamma_base)


def test_workload_like_problem_is_full_rank():
    assert collinear.check(problem()).sum() == 0
    assert collinear.check(problem(1)).sum() == 0


def test_flags_land_in_their_blocks():
    pr = problem(1)
    pr.X[:, 3] = pr.X[:, 1] - 2 * pr.X[:, 2]
    pr.Y[:, 2, 1] = 0.5 * pr.Y[:, 2, 0]
    pr.Y[:, 0, 1] = pr.Y[:, 0, 0]
    pr.Z[:, :, 1] = pr.Z[:, :1, 1] + 3.0  # no variation over the alternatives
    flags = collinear.check(pr)
    p, K, d = pr.p, pr.K, pr.d
    assert flags[:p].tolist() == [0, 0, 0, 1]
    assert flags[p + 2 * d:p + 3 * d].tolist() == [0, 1]
    assert flags[p:p + d].tolist() == [0, 1]
    assert flags[p + K * d:].tolist() == [0, 1, 0]
    assert flags.sum() == 4
    pr.gamma_base = 0
    f0 = collinear.check(pr)
    assert f0[p:p + d].tolist() == [0, 0] and f0.sum() == 3


def test_z_difference_block_is_the_stacked_normalized_z():
    pr = problem()
    Dz = collinear.z_differences(pr)
    i, k, j = 17, 3, 2
    assert Dz.shape == (pr.N * (pr.K - 1), pr.f)
    assert Dz[i * (pr.K - 1) + (k - 1), j] == np.float64(pr.Z[i, k, j]) - np.float64(pr.Z[i, 0, j])


def test_theta_mask_layout():
    pr = problem(1)
    flags = np.zeros(pr.p + pr.K * pr.d + pr.f, dtype=np.int32)
    flags[2] = 1                      # X column 2: beta_k[2] for k = 1..K-1
    flags[pr.p + 0 * pr.d + 1] = 1    # Y_0 column 1: gamma_0[1]
    flags[pr.p + 3 * pr.d + 0] = 1    # Y_3 column 0: gamma_3[0]
    flags[pr.p + pr.K * pr.d + 2] = 1  # alpha[2]
    m = collinear.theta_mask(pr, flags)
    assert m.size == pr.n_theta
    want = set((k - 1) * pr.p + 2 for k in range(1, pr.K))
    g0 = (pr.K - 1) * pr.p
    want |= {g0 + 0 * pr.d + 1, g0 + 3 * pr.d + 0, pr.n_theta - pr.f + 2}
    assert set(np.flatnonzero(m).tolist()) == want
