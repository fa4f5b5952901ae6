"""Batched fits (many uneven problems, one grouped launch per Newton phase) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

THETA_TOL = 1e-6


@pytest.fixture(scope="module")
def cls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300.api import MNLBatch
    return MNLBatch


def uneven_problems(count, seed):
    """Shapes like the batched workload (N log-uniform, K, p, f uniform), scaled down."""
    rng = np.random.default_rng(seed)
    probs = []
    for b in range(count):
        N = int(math.exp(rng.uniform(math.log(300), math.log(6000))))
        K = int(rng.integers(2, 13))
        p = int(rng.integers(1, 11))
        d = int(rng.integers(0, 3))
        f = int(rng.integers(0, 4))
        probs.append(datagen.make_problem(N, K, p, d, f, seed * 1000 + b, intercept=bool(b % 2),
                                          theta_sd=0.4 / math.sqrt(p)))
    return probs


def to_dev(prob):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a.size else None  # noqa: E731
    return dict(X=t(prob.X), Y=t(prob.Y), Z=t(prob.Z), choice=torch.from_numpy(prob.choice).cuda(), K=prob.K)


@pytest.fixture(scope="module")
def batch_and_ref():
    probs = uneven_problems(24, 5)
    refs = [oracle.fit(p)[0] for p in probs]
    return probs, refs


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16"])
def test_batched_fit_matches_oracle_per_problem(cls, batch_and_ref, prec):
    probs, refs = batch_and_ref
    with cls([to_dev(p) for p in probs], precision=prec) as b:
        th, summary, per, rc = b.fit()
        parts = [t.cpu().numpy() for t in b.split(th)]
    assert rc == 0, (summary, per)
    assert summary["converged"] == len(probs)
    for i, (got, ref) in enumerate(zip(parts, refs)):
        err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= THETA_TOL, (prec, i, err, per[i])


def test_result_is_the_same_alone_and_in_the_mix(cls, batch_and_ref):
    probs, refs = batch_and_ref
    k = 7
    with cls([to_dev(probs[k])], precision="bf16") as b:
        alone = b.fit()[0].cpu().numpy()
    with cls([to_dev(p) for p in probs], precision="bf16") as b:
        th = b.fit()[0]
        mixed = b.split(th)[k].cpu().numpy()
    assert np.abs(alone - mixed).max() <= THETA_TOL * np.abs(refs[k]).max()


def test_a_failing_problem_does_not_affect_the_others(cls, batch_and_ref):
    from paper_1404_3177_gb300._native import MNL_ERR_NOT_PD
    probs, refs = batch_and_ref
    bad = datagen.make_problem(800, 4, 3, 0, 0, 77)
    bad.X[:, 2] = 0.0
    members = [probs[0], bad, probs[1]]
    with cls([to_dev(p) for p in members], precision="bf16") as b:
        th, summary, per, rc = b.fit()
        parts = [t.cpu().numpy() for t in b.split(th)]
    assert per[1]["status"] == MNL_ERR_NOT_PD and rc == MNL_ERR_NOT_PD
    for i, ref in ((0, refs[0]), (2, refs[1])):
        assert per[i]["status"] == 0
        assert np.abs(parts[i] - ref).max() / np.abs(ref).max() <= THETA_TOL
