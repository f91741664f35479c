"""Parity at the full workload sizes, in the launch configuration the benchmark
times (default batched plan: persistent grid, CUDA graph), on outputs sampled
across the batch and computed one by one by the CPU oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import kalman
from paper_2510_11077_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def argus():
    from paper_2510_11077_gb300 import argus as a
    a.load()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return a


def _err_ll(ll, ref):
    return (np.abs(ll - ref) / np.maximum(np.abs(ref), 1.0)).max()


def _err_g(g, ref):
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=1, keepdims=True))
    return (np.abs(g - ref) / scale).max()


def _sample(B, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, B - 1], rng.choice(B, k, replace=False)]))


def test_single_pulsar_1000_toas(argus):
    w = inputs.WORKLOADS["psr1_toa1000"]
    data = inputs.make_workload_array(w.name)
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    arr = argus.argus_array_create(data)
    ll = argus.argus_loglik(arr, torch.from_numpy(theta).cuda()).cpu().numpy()
    assert _err_ll(ll, kalman.loglik(data, theta)) <= 1e-9


def test_array20_loglik_4096_walkers(argus):
    w = inputs.WORKLOADS["psr20_toa500-2000_w4096"]
    data = inputs.make_workload_array(w.name)
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    arr = argus.argus_array_create(data)
    ll = argus.argus_loglik(arr, torch.from_numpy(theta).cuda()).cpu().numpy()
    idx = _sample(w.batch, 30, 1)
    assert _err_ll(ll[idx], kalman.loglik(data, theta[idx])) <= 1e-9


def test_array67_grad_1024_walkers(argus):
    w = inputs.WORKLOADS["psr67_toa5000_w1024"]
    data = inputs.make_workload_array(w.name)
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    arr = argus.argus_array_create(data)
    ll, g = argus.argus_loglik_grad(arr, torch.from_numpy(theta).cuda())
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    idx = _sample(w.batch, 2, 2)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert _err_ll(ll[idx], ll_ref) <= 1e-9
    assert _err_g(g[idx], g_ref) <= 1e-6
    # central differences of the GPU log-likelihood for one walker
    th0 = theta[idx[1]]
    D = data.dim
    h = np.array([1e-7] + [1e-4] * (D - 1))
    rows = []
    for j in range(D):
        for s in (1, -1):
            x = th0.copy(); x[j] += s * h[j]; rows.append(x)
    llf = argus.argus_loglik(arr, torch.from_numpy(np.array(rows)).cuda()).cpu().numpy()
    fd = (llf[0::2] - llf[1::2]) / (2 * h)
    assert _err_g(g[idx[1]][None, :], fd[None, :]) <= 1e-4


def test_array100_grad_16384_walkers(argus, tmp_path):
    """In the benchmark's own launch configuration: the autotuner's plan for this
    array and batch (from the committed cache, else tuned here)."""
    from paper_2510_11077_gb300 import autotune
    w = inputs.WORKLOADS["psr100_toalognormal_w16384"]
    data = inputs.make_workload_array(w.name)
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    arr = argus.argus_array_create(data)
    cache = autotune.load_cache()
    key = autotune.plan_key(data.n_toa, w.batch, True, torch.cuda.get_device_name(0))
    if key in cache:
        arr.set_plan(**cache[key]["plan"])
    else:
        arr.set_plan(tape_cache=1, walkers_per_cta=64, ctas_per_sm=8)
    ll, g = argus.argus_loglik_grad(arr, torch.from_numpy(theta).cuda())
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    idx = _sample(w.batch, 1, 3)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert _err_ll(ll[idx], ll_ref) <= 1e-9
    assert _err_g(g[idx], g_ref) <= 1e-6
