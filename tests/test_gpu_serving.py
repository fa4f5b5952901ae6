"""Serving loop (continuous batching) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

THETA_TOL = 1e-6


@pytest.fixture(scope="module")
def Server():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    from paper_1404_3177_gb300.api import MNLServer
    return MNLServer


def requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        N = int(math.exp(rng.uniform(math.log(400), math.log(5000))))
        K = int(rng.integers(3, 12))
        p = int(rng.integers(2, 9))
        f = int(rng.integers(0, 4))
        out.append(datagen.make_problem(N, K, p, 0, f, seed * 1000 + b, intercept=False,
                                        theta_sd=0.5 / math.sqrt(p)))
    return out


def submit(srv, pr):
    return srv.submit(X=pr.X, Y=None, Z=pr.Z if pr.f else None, choice=pr.choice, K=pr.K)


def run_until_done(srv, tickets, arrivals=None, budget=None):
    """Steps the server; arrivals: {tick: [problems]} submitted at that tick."""
    results, pending, tick = {}, dict(tickets), 0
    while True:
        for pr in (arrivals or {}).pop(tick, []):
            pending[submit(srv, pr)] = pr
        active, queued = srv.step()
        if budget is not None:
            assert srv.memory_in_use() <= budget
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                results[t] = (pending.pop(t), r)
        tick += 1
        if not pending and not arrivals and active == 0 and queued == 0:
            return results
        assert tick < 500


@pytest.fixture(scope="module")
def reqs_and_ref():
    reqs = requests(16, 9)
    return reqs, [oracle.fit(r)[0] for r in reqs]


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_served_results_match_oracle(Server, reqs_and_ref, prec):
    reqs, refs = reqs_and_ref
    with Server(precision=prec, mem_budget=8 << 30) as srv:
        tickets = {submit(srv, r): r for r in reqs}
        res = run_until_done(srv, tickets)
    order = {id(r): i for i, r in enumerate(reqs)}
    for t, (pr, (theta, info)) in res.items():
        ref = refs[order[id(pr)]]
        assert info["status"] == 0, info
        assert np.abs(theta - ref).max() / np.abs(ref).max() <= THETA_TOL, (prec, info)


def test_same_result_alone_and_in_the_mix(Server, reqs_and_ref):
    reqs, refs = reqs_and_ref
    k = 3
    with Server(precision="bf16", mem_budget=4 << 30) as srv:
        alone = run_until_done(srv, {submit(srv, reqs[k]): reqs[k]})
    (_, (th_alone, _)), = alone.values()
    # the same request arrives while others are on the device and more arrive after it
    arrivals = {0: reqs[:3], 1: [reqs[k]], 2: reqs[4:10], 4: reqs[10:]}
    with Server(precision="bf16", mem_budget=4 << 30) as srv:
        res = run_until_done(srv, {}, arrivals=arrivals)
    th_mix = next(th for pr, (th, _) in res.values() if pr is reqs[k])
    assert np.abs(th_alone - th_mix).max() <= THETA_TOL * np.abs(refs[k]).max()


def test_admission_respects_the_memory_budget(Server, reqs_and_ref):
    reqs, refs = reqs_and_ref
    budget = 12 << 20  # a few requests at a time
    with Server(precision="bf16", mem_budget=budget) as srv:
        tickets = {submit(srv, r): r for r in reqs}
        res = run_until_done(srv, tickets, budget=budget)
    assert len(res) == len(reqs)
    infos = [info for _, (_, (_, info)) in res.items()]
    assert all(info["status"] == 0 for info in infos)
    assert max(info["queue_ms"] for info in infos) > max(min(info["queue_ms"] for info in infos), 0.0)


def test_request_larger_than_the_budget_is_rejected(Server):
    from paper_1404_3177_gb300._native import MnlError, MNL_ERR_OOM
    pr = datagen.make_problem(200000, 20, 30, 0, 2, 1)
    with Server(precision="bf16", mem_budget=16 << 20) as srv:
        with pytest.raises(MnlError) as e:
            submit(srv, pr)
        assert e.value.status == MNL_ERR_OOM


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_large_request_in_the_mix(Server, reqs_and_ref, prec):
    """n_theta = 1450: solved by the multi-SM path while small requests use one CTA each."""
    reqs, refs = reqs_and_ref
    big = datagen.make_problem(6000, 30, 50, 0, 0, 4242, intercept=True, theta_sd=0.3 / math.sqrt(50))
    assert big.n_theta > 1400
    ref_big = oracle.fit(big)[0]
    with Server(precision=prec, mem_budget=8 << 30) as srv:
        tickets = {submit(srv, r): r for r in reqs[:3] + [big]}
        res = run_until_done(srv, tickets)
    for _, (pr, (theta, info)) in res.items():
        ref = ref_big if pr is big else refs[reqs.index(pr)]
        assert info["status"] == 0, info
        assert np.abs(theta - ref).max() / np.abs(ref).max() <= THETA_TOL


def test_workload5_large_request_in_a_mix_of_small_ones(Server, reqs_and_ref):
    """A large serving request at its full size (N=100000, K=60, p=60, f=4: n_theta = 3544) admitted with small
    ones.  The small results are compared with oracle fits; for the large one an oracle fit takes too long, so
    its estimate theta is checked through the oracle's gradient there: one Newton correction
    d = (-H(theta))^-1 g_oracle(theta), with the GPU's Hessian at theta (pinned to 2e-3 elsewhere), estimates
    theta_hat - theta to within that relative error, so max|d| / max|theta| <= 1e-6 is the coefficient bar."""
    from paper_1404_3177_gb300.api import MNL
    reqs, refs = reqs_and_ref
    big = datagen.config5_large(0)
    assert big.n_theta == 3544
    with Server(precision="bf16", mem_budget=80 << 30) as srv:
        tickets = {submit(srv, r): r for r in reqs[:6] + [big]}
        res = run_until_done(srv, tickets)
    theta_big = None
    for _, (pr, (theta, info)) in res.items():
        assert info["status"] == 0, info
        if pr is big:
            theta_big = theta
            continue
        ref = refs[reqs.index(pr)]
        assert np.abs(theta - ref).max() / np.abs(ref).max() <= THETA_TOL
    _, g = oracle.loglik_grad(big, theta_big)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a.size else None  # noqa: E731
    with MNL(X=d(big.X), Z=d(big.Z), choice=torch.from_numpy(big.choice).cuda(), K=big.K, precision="bf16") as m:
        H = m.hessian(torch.from_numpy(theta_big).cuda()).cpu().numpy()
    corr = np.linalg.solve(-H, g)
    assert np.abs(corr).max() / np.abs(theta_big).max() <= THETA_TOL
