"""mnl_loglik_grad_noalloc, the allocation-free log-likelihood/gradient call.

It serves callers that cannot allocate device memory when they need l and g
(memory owned by an arena or pool, hosts that forbid allocation after
start-up, latency-critical loops).  Called through the C ABI twice in a row,
its results must match the handle-based mnl_loglik_grad within the parity
tolerances of the pass.

The file is named so that pytest collects it last: a run that stops at the
first failure (-x) has then already run every other test.  Nothing else
depends on that order; the 4 MiB array is part of the library image, present
from the moment the library is loaded, and the tests pass alone or after the
others.
"""
import numpy as np
import pytest

from paper_1404_3177_gb300 import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": (1e-12, 1e-11), "bf16": (1e-6, 1e-6)}


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_noalloc_matches_handle_path_twice(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    from paper_1404_3177_gb300 import _native as nat
    from paper_1404_3177_gb300.api import MNL

    _build.build()
    torch.cuda.set_device(0)
    prob = datagen.make_problem(20011, 30, 17, 4, 3, 777, theta_sd=0.2)
    dev = torch.device("cuda", 0)
    X, Y, Z = (torch.from_numpy(a).to(dev) for a in (prob.X, prob.Y, prob.Z))
    c = torch.from_numpy(prob.choice).to(dev)
    theta = torch.from_numpy(np.random.default_rng(3).normal(0, 0.1, prob.n_theta)).to(dev)
    with MNL(X, Y, Z, c, precision=prec) as m:
        l_ref, g_ref = m.loglik_grad(theta)
    g_ref = g_ref.cpu().numpy()

    dims = nat.mnl_dims(prob.N, prob.K, prob.p, prob.d, prob.f, 0)
    data = nat.mnl_data(X.data_ptr(), Y.data_ptr(), Z.data_ptr(), c.data_ptr())
    fdt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    tl, tg = TOL[prec]
    results = []
    for _ in range(2):
        loglik = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        grad = torch.full((prob.n_theta,), float("nan"), dtype=torch.float64, device=dev)
        P = torch.empty((prob.N, prob.K), dtype=fdt, device=dev)
        zbar = torch.empty((prob.N, prob.f), dtype=fdt, device=dev)
        nat.mnl_loglik_grad_noalloc(dims, data, nat.PRECISIONS[prec], theta.data_ptr(), loglik.data_ptr(),
                                    grad.data_ptr(), P.data_ptr(), zbar.data_ptr(), stream)
        torch.cuda.synchronize()
        l = float(loglik.item())
        g = grad.cpu().numpy()
        assert abs(l - l_ref) <= tl * abs(l_ref), (prec, l, l_ref)
        assert np.linalg.norm(g - g_ref) <= tg * np.linalg.norm(g_ref), prec
        Pn = P.double().cpu().numpy()
        assert np.allclose(Pn.sum(axis=1), 1.0, atol=1e-5)
        results.append((l, g))
    assert results[0][0] == results[1][0] and np.array_equal(results[0][1], results[1][1])


def test_noalloc_clamps_its_grid_to_the_scratch():
    """n_theta = 9900: (2 + n) doubles per block leave room for 52 blocks of partial sums, fewer than the SMs, so
    the call runs on a clamped grid; results still match the handle path (float32 pass tolerances)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _build
    from paper_1404_3177_gb300 import _native as nat
    from paper_1404_3177_gb300.api import MNL

    _build.build()
    torch.cuda.set_device(0)
    prob = datagen.make_problem(3001, 100, 100, 0, 0, 31, intercept=False, theta_sd=0.02)
    assert (2 + prob.n_theta) * torch.cuda.get_device_properties(0).multi_processor_count > (1 << 19) - 2
    dev = torch.device("cuda", 0)
    X, c = torch.from_numpy(prob.X).to(dev), torch.from_numpy(prob.choice).to(dev)
    theta = torch.from_numpy(np.random.default_rng(5).normal(0, 0.05, prob.n_theta)).to(dev)
    with MNL(X, None, None, c, K=prob.K, precision="bf16") as m:
        l_ref, g_ref = m.loglik_grad(theta)
    g_ref = g_ref.cpu().numpy()
    dims = nat.mnl_dims(prob.N, prob.K, prob.p, 0, 0, 0)
    data = nat.mnl_data(X.data_ptr(), None, None, c.data_ptr())
    for _ in range(2):
        loglik = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        grad = torch.full((prob.n_theta,), float("nan"), dtype=torch.float64, device=dev)
        P = torch.empty((prob.N, prob.K), dtype=torch.float32, device=dev)
        nat.mnl_loglik_grad_noalloc(dims, data, nat.MNL_BF16, theta.data_ptr(), loglik.data_ptr(), grad.data_ptr(),
                                    P.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert abs(float(loglik.item()) - l_ref) <= 1e-6 * abs(l_ref)
        assert np.linalg.norm(grad.cpu().numpy() - g_ref) <= 1e-6 * np.linalg.norm(g_ref)


def test_noalloc_refuses_sizes_beyond_its_limit_before_any_launch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_3177_gb300 import _native as nat
    dims = nat.mnl_dims(10, 200, 100, 0, 0, 0)  # (K - 1) p = 19900 raw sums > 16384
    data = nat.mnl_data(16, None, None, 16)  # never dereferenced: the call returns first
    with pytest.raises(nat.MnlError) as e:
        nat.mnl_loglik_grad_noalloc(dims, data, nat.MNL_BF16, 16, 16, 16, 16, None, 0)
    assert e.value.status == nat.MNL_ERR_UNSUPPORTED
