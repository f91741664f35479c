"""GPU parity of the continuous wave's pulsar term (ARGUS_PULSAR_TERM) against
the CPU oracle, through the C ABI.  The filter kernels are those of the
Earth-term model; K1 folds the pulsar term into the lane amplitudes and K4
carries the gradient back through the fold.  Tolerances as everywhere:
log-likelihood |d| <= 1e-9 max(|ll|, 1); gradient |d_i| <= 1e-6 max(|g_i|,
1e-3 max_j |g_j|).
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


def pt_data(sizes, seed, model="rw", equad=1e-8):
    return inputs.make_array(np.array(sizes), seed=seed, equad=equad, model=model, pulsar_term=True)


def test_handle_reports_flags_and_dim(argus):
    arr = argus.argus_array_create(pt_data([10, 20, 30], seed=300, model="ou"))
    assert arr.model == argus.ARGUS_NOISE_OU | argus.ARGUS_PULSAR_TERM and arr.dim == 7 + 4 * 3


@pytest.mark.parametrize("model", ["rw", "ou"])
@pytest.mark.parametrize("kind", ["posterior", "prior"])
def test_parity_ragged(argus, model, kind):
    data = pt_data(RAGGED, seed=301, model=model)
    theta = inputs.make_theta_batch(data, 140, seed=7, kind=kind)
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    assert ll_err(ll, kalman.loglik(data, theta)) <= LL_TOL
    idx = np.array([0, 1, 63, 64, 139])
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll[idx], ll_ref) <= LL_TOL
    assert g_err(g[idx], g_ref) <= G_TOL


def test_gradient_vs_central_differences_of_gpu_loglik(argus):
    data = pt_data([400, 250, 330], seed=302)
    theta0 = inputs.make_theta_batch(data, 1, seed=12)[0]
    arr = argus.argus_array_create(data)
    _, g = run(argus, arr, theta0[None, :], grad=True)
    D, k = data.dim, data.n_per_pulsar
    # the lag W d (1 - n.c)/c is ~1e3-1e4 rad: f, the sky position and d need small steps
    steps = np.full(D, 1e-4)
    steps[[0, 4, 5]] = 1e-8
    steps[7 + k - 1::k] = 1e-8
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


def test_zero_distance_cancels_the_wave(argus):
    data = pt_data([300, 120], seed=303)
    theta = inputs.make_theta_batch(data, 40, seed=3)
    theta[:, 9::3] = 1e-15                 # d_p
    nosig = inputs.ArrayData(off=data.off, t=data.t, r=data.r, sigma=data.sigma, pos=data.pos,
                             equad=data.equad, p0=data.p0, theta_true=data.theta_true)
    th0 = np.concatenate([theta[:, :7]] + [theta[:, 7 + 3 * p: 9 + 3 * p] for p in range(2)], axis=1)
    th0[:, 6] = -40.0
    ll = run(argus, argus.argus_array_create(data), theta)
    ll0 = run(argus, argus.argus_array_create(nosig), th0)
    assert ll_err(ll, ll0) <= 1e-12


def test_out_of_domain_distance(argus):
    data = pt_data([30, 60], seed=304, model="ou")
    theta = inputs.make_theta_batch(data, 4, seed=2)
    theta[0, 10] = 0.0       # d of pulsar 0
    theta[1, 14] = -1.0      # d of pulsar 1
    ll, g = run(argus, argus.argus_array_create(data), theta, grad=True)
    assert np.all(np.isneginf(ll[:2])) and np.all(g[:2] == 0.0)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[2:])
    assert ll_err(ll[2:], ll_ref) <= LL_TOL and g_err(g[2:], g_ref) <= G_TOL


def test_plain_host_and_noalloc_paths_agree_bitwise(argus):
    data = pt_data([300, 20, 150], seed=305, model="ou")
    theta = inputs.make_theta_batch(data, 70, seed=10)
    arr = argus.argus_array_create(data)
    ll_b, g_b = run(argus, arr, theta, grad=True)
    ll_h, g_h = argus.argus_loglik_grad(arr, theta)
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
    w = inputs.WORKLOADS["psr20_toa500-2000_w4096"]
    data = inputs.make_workload_array(w.name, pulsar_term=True)
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    idx = np.unique(np.concatenate([[0, w.batch - 1], np.random.default_rng(5).choice(w.batch, 3)]))
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll[idx], ll_ref) <= LL_TOL
    assert g_err(g[idx], g_ref) <= G_TOL
