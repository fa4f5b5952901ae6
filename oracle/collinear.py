"""Collinearity check of the data blocks (Sec. 2.3 `linDepTol`; App. B).

TEST INFRASTRUCTURE ONLY: the tests and the smoke check use this module; the
library's product path never imports it.

The paper asks for a model matrix whose Hessian can be non-singular (App. B):
  1. X and every Y_k have full column rank;
  2. the generic variables Z have linearly independent columns (the paper
     checks the columns of the stacked Z_k, k = 1..K-1, which in its
     normalized form are Z_ik - Z_i0).
The package checks these with R's `qr(tol = linDepTol)` and drops columns of a
collinear set one by one until the rest is linearly independent.

This oracle restates that test as its definition: the columns of a block are
taken in order, and column j is "dependent" when the part of it orthogonal to
the span of the earlier columns that were kept has a norm of at most
tol * ||column j||; dependent columns are dropped and do not enter the span.
The projection is classical Gram-Schmidt applied twice (re-orthogonalization),
in float64, on the float32 data promoted to float64.

Blocks (and the layout of the returned flag vector, length p + K*d + f):
  * X (N x p): flags[0:p];
  * Y_k (N x d) for each alternative k: flags[p + k*d : p + (k+1)*d]; Y_0 is
    checked only when gamma_0 is estimated (gamma_base = 1), else its flags
    are 0;
  * Z: the (N*(K-1)) x f matrix of rows Z_ik - Z_i0, i = 0..N-1, k = 1..K-1:
    flags[p + K*d : p + K*d + f].
Observation weights play no part (the check is on the data).
"""
from __future__ import annotations

import numpy as np


def dependent_columns(M: np.ndarray, tol: float) -> np.ndarray:
    """0/1 flags of the columns of M (rows x cols) that depend on the kept earlier columns."""
    A = np.asarray(M, dtype=np.float64)
    ncol = A.shape[1]
    flags = np.zeros(ncol, dtype=np.int32)
    Q = np.empty((A.shape[0], ncol))  # orthonormal basis of the kept columns: Q[:, :kept]
    kept = 0
    for j in range(ncol):
        a = A[:, j]
        norm_a = np.sqrt(a @ a)
        r = a.copy()
        for _ in range(2):
            r = r - Q[:, :kept] @ (Q[:, :kept].T @ r)
        norm_r = np.sqrt(r @ r)
        if norm_a == 0.0 or norm_r <= tol * norm_a:
            flags[j] = 1
            continue
        Q[:, kept] = r / norm_r
        kept += 1
    return flags


def z_differences(prob) -> np.ndarray:
    """The stacked generic-variable block: rows Z_ik - Z_i0 for k = 1..K-1 ((N*(K-1)) x f)."""
    Z = np.asarray(prob.Z, dtype=np.float64)
    return (Z[:, 1:, :] - Z[:, :1, :]).reshape(-1, prob.f)


def check(prob, tol: float = 1e-6) -> np.ndarray:
    """Flags of the dependent data columns, layout [X (p) | Y_0..Y_{K-1} (K*d) | Z (f)]."""
    p, d, f, K = prob.p, prob.d, prob.f, prob.K
    flags = np.zeros(p + K * d + f, dtype=np.int32)
    if p:
        flags[:p] = dependent_columns(prob.X, tol)
    if d:
        Y = np.asarray(prob.Y, dtype=np.float64)
        for k in range(0 if prob.gamma_base else 1, K):
            flags[p + k * d:p + (k + 1) * d] = dependent_columns(Y[:, k, :], tol)
    if f:
        flags[p + K * d:] = dependent_columns(z_differences(prob), tol)
    return flags


def theta_mask(prob, flags: np.ndarray) -> np.ndarray:
    """1 for each coefficient (eq. "theta vec" order) that belongs to a dropped column:
    beta_k[j] for every k >= 1 when X column j is dropped, gamma_k[j] when column j of Y_k is dropped,
    alpha[j] when Z column j is dropped."""
    p, d, f, K = prob.p, prob.d, prob.f, prob.K
    kg = K if prob.gamma_base else K - 1
    out = []
    for _k in range(1, K):
        out.extend(flags[:p])
    for k in range(0 if prob.gamma_base else 1, K):
        out.extend(flags[p + k * d:p + (k + 1) * d])
    out.extend(flags[p + K * d:p + K * d + f])
    m = np.asarray(out, dtype=np.int32)
    assert m.size == (K - 1) * p + kg * d + f
    return m
