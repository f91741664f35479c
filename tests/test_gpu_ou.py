"""GPU parity of the Ornstein-Uhlenbeck red-noise model (paper, Functionality:
OU processes for pulsar-intrinsic red noise) against the CPU oracle, through
the C ABI.  Same tolerances as the random-walk model: log-likelihood
|d| <= 1e-9 max(|ll|, 1); gradient |d_i| <= 1e-6 max(|g_i|, 1e-3 max_j |g_j|).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import kalman
from paper_2510_11077_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LL_TOL = 1e-9
G_TOL = 1e-6
RAGGED = [1, 37, 200, 513, 129]


@pytest.fixture(scope="module")
def argus():
    from paper_2510_11077_gb300 import argus as a
    a.load()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return a


def ll_err(ll, ref):
    ll, ref = np.asarray(ll), np.asarray(ref)
    both_inf = np.isneginf(ll) & np.isneginf(ref)
    with np.errstate(invalid="ignore"):
        d = np.where(both_inf, 0.0, np.abs(ll - ref) / np.maximum(np.abs(ref), 1.0))
    return np.nan_to_num(d, nan=np.inf).max()


def g_err(g, ref):
    g, ref = np.atleast_2d(g), np.atleast_2d(ref)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=1, keepdims=True))
    scale = np.where(scale == 0, 1.0, scale)
    return np.nan_to_num(np.abs(g - ref) / scale, nan=np.inf).max()


def run(argus, arr, theta, grad=False):
    th = torch.from_numpy(np.ascontiguousarray(theta)).cuda()
    if grad:
        ll, g = argus.argus_loglik_grad(arr, th)
        return ll.cpu().numpy(), g.cpu().numpy()
    return argus.argus_loglik(arr, th).cpu().numpy()


def ou_data(sizes, seed, equad=1e-8):
    return inputs.make_array(np.array(sizes), seed=seed, equad=equad, model="ou")


def test_handle_reports_model_and_dim(argus):
    data = ou_data([10, 20, 30], seed=200)
    arr = argus.argus_array_create(data)
    assert arr.noise_model == argus.ARGUS_NOISE_OU and arr.dim == 7 + 3 * 3


@pytest.mark.parametrize("kind", ["posterior", "prior"])
def test_loglik_parity_ragged(argus, kind):
    data = ou_data(RAGGED + [1000], seed=201)
    theta = inputs.make_theta_batch(data, 300, seed=5, kind=kind)
    arr = argus.argus_array_create(data)
    assert ll_err(run(argus, arr, theta), kalman.loglik(data, theta)) <= LL_TOL


@pytest.mark.parametrize("kind", ["posterior", "prior"])
@pytest.mark.parametrize("tape_cache", [0, 1])
def test_grad_parity_ragged(argus, kind, tape_cache):
    data = ou_data(RAGGED, seed=202, equad=2e-8)
    theta = inputs.make_theta_batch(data, 140, seed=7, kind=kind)
    arr = argus.argus_array_create(data)
    arr.set_plan(tape_cache=tape_cache)
    ll, g = run(argus, arr, theta, grad=True)
    idx = np.array([0, 1, 63, 64, 127, 128, 139])
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll, kalman.loglik(data, theta)) <= LL_TOL
    assert ll_err(ll[idx], ll_ref) <= LL_TOL
    assert g_err(g[idx], g_ref) <= G_TOL


@pytest.mark.parametrize("stride", [1, 7, 0])
def test_grad_checkpoint_strides(argus, stride):
    data = ou_data([49, 50, 64, 3], seed=203)
    theta = inputs.make_theta_batch(data, 40, seed=8, kind="prior")
    arr = argus.argus_array_create(data)
    arr.set_plan(ckpt_stride=stride)
    ll, g = run(argus, arr, theta, grad=True)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[:6])
    assert ll_err(ll[:6], ll_ref) <= LL_TOL
    assert g_err(g[:6], g_ref) <= G_TOL


@pytest.mark.parametrize("log10_gamma", [-12.0, -7.0, -6.0, -4.5])
def test_steps_across_the_series_switch(argus, log10_gamma):
    """gamma dt spread across the 1/64, 1/8 and 1/2 boundaries of the
    transition's series and beyond (down to a ~ e^-100)."""
    rng = np.random.default_rng(int(-10 * log10_gamma))
    gaps = np.concatenate([rng.uniform(1e3, 1e5, 60), rng.uniform(1e5, 3e6, 60),
                           rng.uniform(3e6, 3e7, 40)])
    rng.shuffle(gaps)
    t = np.concatenate([[0.0], np.cumsum(gaps)])
    n = len(t)
    data = inputs.ArrayData(off=np.array([0, n]), t=t, r=1e-6 * rng.standard_normal(n),
                            sigma=np.full(n, 1e-7), pos=np.array([[0.0, 0.6, 0.8]]),
                            equad=np.array([1e-8]), p0=np.array([inputs.P0_DEFAULT]),
                            theta_true=np.zeros(10), model="ou")
    theta = np.tile(np.array([-8.3, 0.5, 0.4, 0.2, 0.1, 1.0, -13.5, -19.5, log10_gamma, 1.05]), (70, 1))
    theta[:, 8] += np.linspace(-0.3, 0.3, 70)
    theta[:, 7] += np.linspace(0.2, -0.2, 70)
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    idx = np.array([0, 31, 69])
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll, kalman.loglik(data, theta)) <= LL_TOL
    assert g_err(g[idx], g_ref) <= G_TOL


def test_tiny_gamma_equals_random_walk_on_the_gpu(argus):
    data = ou_data([300, 120, 57], seed=204)
    theta = inputs.make_theta_batch(data, 64, seed=3)
    theta[:, 8::3] = -22.0
    rw = inputs.ArrayData(off=data.off, t=data.t, r=data.r, sigma=data.sigma, pos=data.pos,
                          equad=data.equad, p0=data.p0, theta_true=data.theta_true, model="rw")
    th_rw = np.concatenate([theta[:, :7]] + [theta[:, [7 + 3 * p, 9 + 3 * p]] for p in range(3)], axis=1)
    ll_ou, g_ou = run(argus, argus.argus_array_create(data), theta, grad=True)
    ll_rw, g_rw = run(argus, argus.argus_array_create(rw), th_rw, grad=True)
    assert ll_err(ll_ou, ll_rw) <= 1e-12
    keep = [j for j in range(data.dim) if j < 7 or (j - 7) % 3 != 1]
    assert g_err(g_ou[:, keep], g_rw) <= 1e-9


def test_gamma_gradient_vs_central_differences_of_gpu_loglik(argus):
    data = ou_data([400, 250, 330], seed=205)
    theta0 = inputs.make_theta_batch(data, 1, seed=12)[0]
    arr = argus.argus_array_create(data)
    _, g = run(argus, arr, theta0[None, :], grad=True)
    D = data.dim
    steps = np.array([1e-7] + [1e-4] * (D - 1))
    rows = []
    for j in range(D):
        for h in (steps[j], steps[j] / 2):
            for sgn in (1, -1):
                x = theta0.copy(); x[j] += sgn * h
                rows.append(x)
    ll = run(argus, arr, np.array(rows))
    fd = []
    for j in range(D):
        a = ll[4 * j: 4 * j + 4]
        c1 = (a[0] - a[1]) / (2 * steps[j])
        c2 = (a[2] - a[3]) / steps[j]
        fd.append((4 * c2 - c1) / 3)
    assert g_err(g[0], np.array(fd)) <= 1e-5


def test_out_of_domain_and_empty_pulsar(argus):
    data = ou_data([0, 30, 60], seed=206)
    theta = inputs.make_theta_batch(data, 5, seed=2)
    theta[0, 12] = -1.0     # EFAC < 0 (third noise slot of pulsar 1)
    theta[1, 11] = np.nan   # log10 gamma of pulsar 1
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    assert np.all(np.isneginf(ll[:2])) and np.all(g[:2] == 0.0)
    assert np.all(g[2:, 7:10] == 0.0)           # the empty pulsar has no gradient
    ll_ref, g_ref = kalman.loglik_grad(data, theta[2:])
    assert ll_err(ll[2:], ll_ref) <= LL_TOL and g_err(g[2:], g_ref) <= G_TOL


def test_plain_graph_host_and_noalloc_paths_agree_bitwise(argus):
    data = ou_data([300, 20, 150], seed=207)
    theta = inputs.make_theta_batch(data, 70, seed=10)
    arr = argus.argus_array_create(data)
    ll_b, g_b = run(argus, arr, theta, grad=True)
    ll_h, g_h = argus.argus_loglik_grad(arr, theta)           # host pointers (numpy)
    assert np.array_equal(ll_b, ll_h) and np.array_equal(g_b, g_h)
    th = torch.from_numpy(theta).cuda()
    ll_n = torch.empty(70, dtype=torch.float64, device="cuda")
    g_n = torch.empty((70, data.dim), dtype=torch.float64, device="cuda")
    argus.argus_loglik_grad_noalloc(arr, th, ll_n, g_n)
    assert np.array_equal(ll_b, ll_n.cpu().numpy()) and np.array_equal(g_b, g_n.cpu().numpy())
    arr.set_plan(mode=argus.ARGUS_MODE_PLAIN)
    ll_p, g_p = run(argus, arr, theta, grad=True)
    assert np.array_equal(ll_b, ll_p) and np.array_equal(g_b, g_p)


def test_full_size_array20_4096_walkers(argus):
    """The 20-pulsar workload with OU red noise, at its full batch, in the
    default batched plan; sampled walkers against the oracle."""
    w = inputs.WORKLOADS["psr20_toa500-2000_w4096"]
    data = inputs.make_workload_array(w.name, model="ou")
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    idx = np.unique(np.concatenate([[0, w.batch - 1], np.random.default_rng(4).choice(w.batch, 3)]))
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll[idx], ll_ref) <= LL_TOL
    assert g_err(g[idx], g_ref) <= G_TOL
