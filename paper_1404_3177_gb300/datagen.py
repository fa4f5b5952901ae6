"""Seeded synthetic multinomial-logit problems (inputs only).

This module draws the data blocks of the model of Sec. 2.1 (eq. "unormalized
utility"): individual-specific columns X [N][p], alternative-specific columns
with per-class coefficients Y [N][K][d], alternative-specific columns with a
generic coefficient Z [N][K][f], and the observed choices y [N] (0 = base).

It holds none of the estimation arithmetic (no probabilities, log-likelihood,
gradient or Hessian).  Choices are drawn by the random-utility principle the
paper states in Sec. 2.1: each alternative's observed utility plus i.i.d.
standard Gumbel noise, and the individual picks the arg-max ("Gumbel-max").

Both the FP64 oracle (tests) and the GPU path (tests, bench) receive exactly
the float32 arrays produced here; the oracle promotes them to float64.

Determinism: every block of ``ROW_BLOCK`` observations is drawn from its own
Philox stream keyed by (seed, block index), so results do not depend on how
many rows are generated at once.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ROW_BLOCK = 4096
SEED_BASE = 1404317700


@dataclasses.dataclass
class Problem:
    """One synthetic problem.  Arrays are C-contiguous float32/int32."""

    N: int
    K: int
    p: int
    d: int
    f: int
    gamma_base: int
    X: np.ndarray  # [N][p] float32
    Y: np.ndarray  # [N][K][d] float32
    Z: np.ndarray  # [N][K][f] float32 (raw, not differenced against alternative 0)
    choice: np.ndarray  # [N] int32 in [0, K)
    theta_true: np.ndarray  # [n_theta] float64, layout of eq. "theta vec"
    name: str = ""

    @property
    def n_theta(self) -> int:
        return num_params(self.K, self.p, self.d, self.f, self.gamma_base)

    def input_bytes(self) -> int:
        return self.X.nbytes + self.Y.nbytes + self.Z.nbytes + self.choice.nbytes


def num_params(K: int, p: int, d: int, f: int, gamma_base: int = 0) -> int:
    """Coefficient count: (K-1) beta_k of length p, (K-1) or K gamma_k of length d, one alpha of length f."""
    return (K - 1) * p + (K if gamma_base else K - 1) * d + f


def _block_rng(seed: int, block: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, block, stream])))


def make_problem(
    N: int,
    K: int,
    p: int,
    d: int,
    f: int,
    seed: int,
    *,
    intercept: bool = True,
    theta_sd: float = 0.5,
    sparse_cols: tuple[int, int] | None = None,
    sparse_prob: float = 0.1,
    gamma_base: int = 0,
    theta_true: np.ndarray | None = None,
    name: str = "",
) -> Problem:
    """Draw one problem.

    X column 0 is the intercept (all ones) when ``intercept`` is set; the other
    X columns and all Y, Z entries are iid N(0,1), except X columns in the
    half-open range ``sparse_cols`` which are Bernoulli(``sparse_prob``) 0/1
    indicators.  True coefficients are iid N(0, theta_sd^2) unless given.
    """
    if N < 0 or K < 2 or min(p, d, f) < 0:
        raise ValueError("bad problem dimensions")
    nth = num_params(K, p, d, f, gamma_base)
    if theta_true is None:
        theta_true = _block_rng(seed, 0, 99).normal(0.0, theta_sd, size=nth)
    theta_true = np.ascontiguousarray(theta_true, dtype=np.float64)
    # Coefficient views in the eq. "theta vec" order.
    nb = (K - 1) * p
    beta = np.zeros((K, p))
    beta[1:] = theta_true[:nb].reshape(K - 1, p)
    ng = (K if gamma_base else K - 1) * d
    gamma = np.zeros((K, d))
    if gamma_base:
        gamma[:] = theta_true[nb:nb + ng].reshape(K, d)
    else:
        gamma[1:] = theta_true[nb:nb + ng].reshape(K - 1, d)
    alpha = theta_true[nb + ng:]

    X = np.empty((N, p), np.float32)
    Y = np.empty((N, K, d), np.float32)
    Z = np.empty((N, K, f), np.float32)
    choice = np.empty((N,), np.int32)
    for blk, r0 in enumerate(range(0, N, ROW_BLOCK)):
        r1 = min(N, r0 + ROW_BLOCK)
        n = r1 - r0
        rng = _block_rng(seed, blk, 0)
        xb = rng.standard_normal((n, p))
        if intercept and p > 0:
            xb[:, 0] = 1.0
        if sparse_cols is not None:
            c0, c1 = sparse_cols
            xb[:, c0:c1] = (rng.random((n, c1 - c0)) < sparse_prob).astype(np.float64)
        yb = rng.standard_normal((n, K, d))
        zb = rng.standard_normal((n, K, f))
        X[r0:r1] = xb
        Y[r0:r1] = yb
        Z[r0:r1] = zb
        # Observed utility of every alternative from the stored float32 data
        # (the data-generating process; beta_0 = 0 and, with gamma_base = 0, gamma_0 = 0).
        x32 = X[r0:r1].astype(np.float64)
        util = x32 @ beta.T
        util += np.einsum("nkd,kd->nk", Y[r0:r1].astype(np.float64), gamma)
        util += Z[r0:r1].astype(np.float64) @ alpha if f > 0 else 0.0
        u01 = rng.random((n, K))
        gumbel = -np.log(-np.log(np.clip(u01, 1e-300, None)))
        choice[r0:r1] = np.argmax(util + gumbel, axis=1).astype(np.int32)
    return Problem(N, K, p, d, f, gamma_base, X, Y, Z, choice, theta_true, name)


# ---------------------------------------------------------------------------
# The workloads: five shapes with fixed seeds.
# ---------------------------------------------------------------------------

def config1() -> Problem:
    """N=2000, K=5, X = [1, 3 x N(0,1)] (p=4), Z f=2, Y d=1, theta ~ N(0, 0.5^2); 22 coefficients."""
    return make_problem(2000, 5, 4, 1, 2, SEED_BASE + 1, intercept=True, theta_sd=0.5, name="c1_N2000_K5_p4_d1_f2")


def config2(N: int = 200_000) -> Problem:
    """N=200000, K=50, p=50 (intercept + 49 N(0,1)), f=5, d=5, theta ~ N(0, 0.3^2/50); 2700 coefficients."""
    return make_problem(N, 50, 50, 5, 5, SEED_BASE + 2, intercept=True, theta_sd=0.3 / math.sqrt(50),
                        name=f"c2_N{N}_K50_p50_d5_f5")


def config3(N: int = 500_000) -> Problem:
    """N=500000, K=100, p=100 (no intercept; columns 70..99 Bernoulli(0.1)), f=10, d=0; 9910 coefficients."""
    return make_problem(N, 100, 100, 0, 10, SEED_BASE + 3, intercept=False, theta_sd=0.2 / math.sqrt(100),
                        sparse_cols=(70, 100), name=f"c3_N{N}_K100_p100_d0_f10")


def config3_shard(rank: int, N: int = 500_000) -> Problem:
    """Rank `rank`'s observations of the observation-sharded workload: the config-3 shape and true coefficients,
    rank 0's rows are config3() itself and every other rank draws its own rows (seed offset by the rank)."""
    if rank == 0:
        return config3(N)
    theta = make_problem(0, 100, 100, 0, 10, SEED_BASE + 3, intercept=False, theta_sd=0.2 / math.sqrt(100)).theta_true
    return make_problem(N, 100, 100, 0, 10, SEED_BASE + 3 + 7919 * rank, intercept=False, sparse_cols=(70, 100),
                        theta_true=theta, name=f"c3_shard{rank}_N{N}_K100_p100_d0_f10")


def config4_shapes(count: int = 2048, seed: int = SEED_BASE + 4) -> list[tuple[int, int, int, int]]:
    """(N, K, p, f) of the batched workload: N log-uniform in [500, 50000], K in 3..30, p in 2..40, f in 0..4, d=0."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 1 << 20])))
    out = []
    for _ in range(count):
        N = int(math.floor(math.exp(rng.uniform(math.log(500), math.log(50000)))))
        K = int(rng.integers(3, 31))
        p = int(rng.integers(2, 41))
        f = int(rng.integers(0, 5))
        out.append((N, K, p, f))
    return out


def config4_problem(b: int, shape: tuple[int, int, int, int], seed: int = SEED_BASE + 4) -> Problem:
    """Problem b of the batched workload (X, Z iid N(0,1), no intercept, theta ~ N(0, 0.5^2/p))."""
    N, K, p, f = shape
    return make_problem(N, K, p, 0, f, seed * 4096 + b, intercept=False, theta_sd=0.5 / math.sqrt(p),
                        name=f"c4_b{b}_N{N}_K{K}_p{p}_f{f}")


def config5_large(r: int, seed: int = SEED_BASE + 5) -> Problem:
    """A large serving request: N=100000, K=60, p=60, f=4, d=0, theta ~ N(0, 0.5^2/60)."""
    return make_problem(100_000, 60, 60, 0, 4, seed * 4096 + r, intercept=False, theta_sd=0.5 / math.sqrt(60),
                        name=f"c5_large_r{r}")


def config5_arrivals(rate: float = 500.0, duration: float = 60.0, large_frac: float = 0.02,
                     seed: int = SEED_BASE + 5) -> list[tuple[float, bool]]:
    """Poisson arrival times (seeded exponential gaps) and whether each request is a large one."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 1 << 21])))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append((t, bool(rng.random() < large_frac)))
