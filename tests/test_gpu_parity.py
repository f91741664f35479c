"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (fixed by the target of the method's GPU port): log-likelihood
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
    th = torch.from_numpy(theta).cuda()
    if grad:
        ll, g = argus.argus_loglik_grad(arr, th)
        torch.cuda.synchronize()
        return ll.cpu().numpy(), g.cpu().numpy()
    ll = argus.argus_loglik(arr, th)
    torch.cuda.synchronize()
    return ll.cpu().numpy()


# ragged array: spans several TOA chunks, several walker tiles, a ragged tail
RAGGED = [1, 37, 200, 513, 1000, 129]


@pytest.mark.parametrize("kind", ["posterior", "prior"])
def test_loglik_parity_ragged(argus, kind):
    data = inputs.make_array(np.array(RAGGED), seed=101, equad=1e-8)
    theta = inputs.make_theta_batch(data, 300, seed=5, kind=kind)
    arr = argus.argus_array_create(data)
    ll = run(argus, arr, theta)
    ref = kalman.loglik(data, theta)
    assert ll_err(ll, ref) <= LL_TOL


def test_lane_loglik_parity(argus):
    data = inputs.make_array(np.array(RAGGED), seed=102)
    theta = inputs.make_theta_batch(data, 130, seed=6)
    arr = argus.argus_array_create(data)
    lane = argus.argus_lane_loglik(arr, torch.from_numpy(theta).cuda()).cpu().numpy()
    _, ref = kalman.loglik(data, theta, lanes=True)
    assert ll_err(lane.ravel(), ref.ravel()) <= LL_TOL


@pytest.mark.parametrize("kind", ["posterior", "prior"])
def test_grad_parity_ragged(argus, kind):
    data = inputs.make_array(np.array([1, 37, 200, 513, 129]), seed=103, equad=2e-8)
    theta = inputs.make_theta_batch(data, 140, seed=7, kind=kind)
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    idx = np.array([0, 1, 63, 64, 127, 128, 139])
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll, kalman.loglik(data, theta)) <= LL_TOL
    assert ll_err(ll[idx], ll_ref) <= LL_TOL
    assert g_err(g[idx], g_ref) <= G_TOL


@pytest.mark.parametrize("stride", [1, 7, 16, 0])
def test_grad_checkpoint_strides(argus, stride):
    """The adjoint does not depend on the checkpoint stride (segment edges at
    N = c^2, c^2 + 1 and a stride of 1 included)."""
    data = inputs.make_array(np.array([49, 50, 64, 3]), seed=104)
    theta = inputs.make_theta_batch(data, 40, seed=8)
    arr = argus.argus_array_create(data)
    arr.set_plan(ckpt_stride=stride)
    ll, g = run(argus, arr, theta, grad=True)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[:6])
    assert ll_err(ll[:6], ll_ref) <= LL_TOL
    assert g_err(g[:6], g_ref) <= G_TOL


def test_edge_cases_empty_single_and_equal_times(argus):
    data = inputs.make_array(np.array([0, 1, 5, 40]), seed=105)
    # equal TOA times inside a pulsar (dt = 0)
    a, b = data.off[3], data.off[4]
    data.t[a + 10:a + 13] = data.t[a + 10]
    data.t[a:b] = np.sort(data.t[a:b])
    theta = inputs.make_theta_batch(data, 33, seed=9)
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[:4])
    assert ll_err(ll[:4], ll_ref) <= LL_TOL
    assert g_err(g[:4], g_ref) <= G_TOL
    lane = argus.argus_lane_loglik(arr, torch.from_numpy(theta).cuda()).cpu().numpy()
    assert np.all(lane[:, 0] == 0.0)           # empty pulsar contributes nothing
    assert np.all(g[:, 7:9] == 0.0)             # ... and has no gradient


def test_batch_sizes_zero_and_one(argus):
    data = inputs.make_array(np.array([30, 60]), seed=106)
    arr = argus.argus_array_create(data)
    empty = np.zeros((0, data.dim))
    out = argus.argus_loglik(arr, torch.from_numpy(empty).cuda())
    assert out.shape == (0,)
    theta = inputs.make_theta_batch(data, 1, seed=1)
    ll, g = run(argus, arr, theta, grad=True)
    ll_ref, g_ref = kalman.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL and g_err(g, g_ref) <= G_TOL


def test_out_of_domain_walkers(argus):
    data = inputs.make_array(np.array([30, 60]), seed=107)
    theta = inputs.make_theta_batch(data, 6, seed=2)
    theta[0, 8] = -1.0      # EFAC < 0
    theta[1, 3] = 1.2       # |cos iota| > 1
    theta[2, 4] = -1.5      # |sin delta| > 1
    theta[3, 0] = np.nan
    theta[4, 10] = np.inf
    arr = argus.argus_array_create(data)
    ll, g = run(argus, arr, theta, grad=True)
    assert np.all(np.isneginf(ll[:5])) and np.isfinite(ll[5])
    assert np.all(g[:5] == 0.0)
    ref = kalman.loglik(data, theta)
    assert ll_err(ll, ref) <= LL_TOL


def test_plain_graph_and_host_paths_agree_bitwise(argus):
    data = inputs.make_array(np.array([300, 20, 150]), seed=108)
    theta = inputs.make_theta_batch(data, 70, seed=10)
    arr = argus.argus_array_create(data)
    ll_b, g_b = run(argus, arr, theta, grad=True)
    ll_b2, g_b2 = run(argus, arr, theta, grad=True)          # graph replay
    assert np.array_equal(ll_b, ll_b2) and np.array_equal(g_b, g_b2)
    ll_h, g_h = argus.argus_loglik_grad(arr, theta)           # host pointers (numpy)
    assert np.array_equal(ll_b, ll_h) and np.array_equal(g_b, g_h)
    for w in (32, 64, 256):
        arr.set_plan(walkers_per_cta=w, use_graph=0, ctas_per_sm=2)
        ll_w, g_w = run(argus, arr, theta, grad=True)
        assert np.array_equal(ll_b, ll_w) and np.array_equal(g_b, g_w)
    arr.set_plan(mode=argus.ARGUS_MODE_PLAIN)
    ll_p, g_p = run(argus, arr, theta, grad=True)
    assert np.array_equal(ll_b, ll_p) and np.array_equal(g_b, g_p)
    ll_pf = run(argus, arr, theta)
    assert np.array_equal(ll_b, ll_pf)


def test_duplicate_walkers_and_pulsar_permutation(argus):
    data = inputs.make_array(np.array([90, 40, 60]), seed=109)
    theta = inputs.make_theta_batch(data, 10, seed=11)
    theta[7] = theta[2]
    arr = argus.argus_array_create(data)
    ll = run(argus, arr, theta)
    assert ll[7] == ll[2]
    perm = [2, 0, 1]
    d2 = inputs.ArrayData(
        off=np.concatenate([[0], np.cumsum(data.n_toa[perm])]),
        t=np.concatenate([data.pulsar(p)[0] for p in perm]),
        r=np.concatenate([data.pulsar(p)[1] for p in perm]),
        sigma=np.concatenate([data.pulsar(p)[2] for p in perm]),
        pos=data.pos[perm], equad=data.equad[perm], p0=data.p0[perm], theta_true=data.theta_true)
    th2 = np.concatenate([theta[:, :7]] + [theta[:, 7 + 2 * p: 9 + 2 * p] for p in perm], axis=1)
    ll2 = run(argus, argus.argus_array_create(d2), th2)
    assert np.allclose(ll, ll2, rtol=1e-13, atol=0)


def test_gradient_vs_central_differences_of_gpu_loglik(argus):
    data = inputs.make_array(np.array([400, 250, 330]), seed=110, equad=1e-8)
    theta0 = inputs.make_theta_batch(data, 1, seed=12)[0]
    arr = argus.argus_array_create(data)
    _, g = run(argus, arr, theta0[None, :], grad=True)
    D = data.dim
    steps = np.array([1e-7] + [1e-4] * (D - 1))
    # Richardson-extrapolated central differences, all in one batch
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


def test_autograd_function(argus):
    data = inputs.make_array(np.array([80, 120]), seed=111)
    theta = inputs.make_theta_batch(data, 5, seed=13)
    arr = argus.argus_array_create(data)
    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    ll = argus.loglik_autograd(th, arr)
    w = torch.arange(1, 6, dtype=torch.float64, device="cuda")
    (ll * w).sum().backward()
    _, g = run(argus, arr, theta, grad=True)
    assert np.allclose(th.grad.cpu().numpy(), w.cpu().numpy()[:, None] * g, rtol=0, atol=0)


def test_repeat_runs_are_deterministic(argus):
    data = inputs.make_array(np.array([500, 700]), seed=112)
    theta = inputs.make_theta_batch(data, 1000, seed=14, kind="prior")
    arr = argus.argus_array_create(data)
    arr.set_plan(use_graph=0)
    a = run(argus, arr, theta, grad=True)
    b = run(argus, arr, theta, grad=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_tape_cache_mode_matches_oracle_and_recompute_mode(argus):
    data = inputs.make_array(np.array([1, 37, 200, 513, 129, 0]), seed=113, equad=1e-8)
    theta = inputs.make_theta_batch(data, 150, seed=15)
    arr = argus.argus_array_create(data)
    ll0, g0 = run(argus, arr, theta, grad=True)
    arr.set_plan(tape_cache=1)
    ll1, g1 = run(argus, arr, theta, grad=True)
    assert ll_err(ll1, ll0) <= 1e-13 and g_err(g1, g0) <= 1e-12
    idx = np.array([0, 77, 149])
    ll_ref, g_ref = kalman.loglik_grad(data, theta[idx])
    assert ll_err(ll1[idx], ll_ref) <= LL_TOL and g_err(g1[idx], g_ref) <= G_TOL


def test_autotuner_picks_and_caches_a_plan(argus, tmp_path):
    from paper_2510_11077_gb300 import autotune
    data = inputs.make_array(np.array([300, 120, 700]), seed=114)
    theta = torch.from_numpy(inputs.make_theta_batch(data, 300, seed=16)).cuda()
    arr = argus.argus_array_create(data)
    cache = str(tmp_path / "plans.json")
    space = {"walkers_per_cta": (64, 128), "ctas_per_sm": (2, 4), "tape_cache": (0, 1)}
    res = autotune.autotune(arr, theta, data.n_toa, grad=True, space=space, cache_path=cache)
    assert not res["cached"] and len(res["tried"]) == 8
    assert arr.get_plan()["walkers_per_cta"] == res["plan"]["walkers_per_cta"]
    arr2 = argus.argus_array_create(data)
    res2 = autotune.autotune(arr2, theta, data.n_toa, grad=True, space=space, cache_path=cache)
    assert res2["cached"] and res2["plan"] == res["plan"]
    ll, g = argus.argus_loglik_grad(arr2, theta)
    ll_ref, g_ref = kalman.loglik_grad(data, theta[:3].cpu().numpy())
    assert ll_err(ll[:3].cpu().numpy(), ll_ref) <= LL_TOL
    assert g_err(g[:3].cpu().numpy(), g_ref) <= G_TOL


def test_cw_signal_matches_oracle(argus):
    from oracle import dense
    data = inputs.make_array(np.array([300, 0, 57, 1000]), seed=115)
    arr = argus.argus_array_create(data)
    for th in inputs.make_theta_batch(data, 3, seed=19, kind="prior"):
        s = argus.argus_cw_signal(arr, th, int(data.off[-1]))
        ref = np.concatenate([dense.cw_signal(th[:7], data.pos[p], data.pulsar(p)[0])
                              for p in range(data.n_pulsars)])
        assert np.max(np.abs(s - ref)) <= 1e-12 * np.max(np.abs(ref))
