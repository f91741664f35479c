"""GPU parity of the joint likelihood with a Hellings-Downs correlated GW
background (include/argus_gwb.h) against the CPU oracle (oracle/gwb.c).
Tolerance as everywhere: |d| <= 1e-9 max(|ll|, 1)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import gwb
from paper_2510_11077_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LL_TOL = 1e-9


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


def thetas(P, B, rng, lh=(-20.5, -18.0), lg=(-10.0, -7.0)):
    th = np.empty((B, 2 + 3 * P))
    th[:, 0] = rng.uniform(*lh, B)
    th[:, 1] = rng.uniform(*lg, B)
    th[:, 2::3] = rng.uniform(-20.8, -19.2, (B, P))
    th[:, 3::3] = rng.uniform(-9.8, -7.2, (B, P))
    th[:, 4::3] = rng.uniform(0.85, 1.15, (B, P))
    return th


def run(argus, arr, theta):
    return argus.argus_gwb_loglik(arr, torch.from_numpy(np.ascontiguousarray(theta)).cuda()).cpu().numpy()


@pytest.mark.parametrize("sizes", [[40], [30, 50, 20], [0, 25, 1, 60], [15] * 8])
def test_parity_small_arrays(argus, sizes):
    data = inputs.make_array(np.array(sizes), seed=500 + len(sizes), equad=1e-8)
    theta = thetas(len(sizes), 24, np.random.default_rng(len(sizes)))
    arr = argus.GwbArray(data)
    assert arr.dim == 2 + 3 * len(sizes)
    assert ll_err(run(argus, arr, theta), gwb.loglik(data, theta)) <= LL_TOL


def test_equal_times_across_pulsars(argus):
    data = inputs.make_array(np.array([40, 35, 25]), seed=501)
    a, b = data.off[1], data.off[2]
    data.t[a:a + 10] = data.t[3:13]                      # pulsar 1 shares ten TOA times with pulsar 0
    data.t[a:b] = np.sort(data.t[a:b])
    data.t[b + 2:b + 5] = data.t[b + 2]                  # and pulsar 2 repeats one of its own
    theta = thetas(3, 16, np.random.default_rng(2))
    arr = argus.GwbArray(data)
    assert ll_err(run(argus, arr, theta), gwb.loglik(data, theta)) <= LL_TOL


def test_twenty_pulsars(argus):
    """20 pulsars (the 60-dimensional joint state of the 20-pulsar workload),
    100 TOAs each so that the oracle's dense algebra finishes in seconds."""
    rng = np.random.default_rng(3)
    data = inputs.make_array(np.full(20, 100), seed=502, equad=1e-8)
    theta = thetas(20, 6, rng)
    arr = argus.GwbArray(data)
    assert ll_err(run(argus, arr, theta), gwb.loglik(data, theta)) <= LL_TOL


def test_largest_supported_array(argus):
    """64 pulsars: the 192-dimensional joint covariance, packed, in shared memory."""
    data = inputs.make_array(np.full(64, 5), seed=503)
    theta = thetas(64, 3, np.random.default_rng(4))
    arr = argus.GwbArray(data)
    assert ll_err(run(argus, arr, theta), gwb.loglik(data, theta)) <= LL_TOL


def test_gradient_of_the_largest_supported_array(argus):
    """48 pulsars, the gradient's limit (covariance and adjoint both packed in
    shared memory); 49 are refused."""
    data = inputs.make_array(np.full(48, 4), seed=515)
    th0 = thetas(48, 1, np.random.default_rng(16), lh=(-19.2, -18.6))[0]
    arr = argus.GwbArray(data)
    ll, g = argus.argus_gwb_loglik_grad(arr, torch.from_numpy(th0[None, :]).cuda())
    ll, g = ll.cpu().numpy(), g.cpu().numpy()[0]
    assert ll_err(ll, gwb.loglik(data, th0[None, :])) <= LL_TOL
    assert ll_err(ll, run(argus, arr, th0[None, :])) <= 1e-13
    # Richardson central differences of the GPU likelihood on the background's
    # parameters and those of the first, a middle and the last pulsar
    js = [0, 1] + [2 + 3 * p + k for p in (0, 23, 47) for k in range(3)]
    rows = []
    for j in js:
        for h in (1e-4, 5e-5):
            for sgn in (1, -1):
                x = th0.copy(); x[j] += sgn * h
                rows.append(x)
    lf = run(argus, arr, np.array(rows))
    fd = np.array([(4 * (lf[4 * i + 2] - lf[4 * i + 3]) / 1e-4 - (lf[4 * i] - lf[4 * i + 1]) / 2e-4) / 3
                   for i in range(len(js))])
    assert g_err(g[js], fd) <= 1e-5
    big = inputs.make_array(np.full(49, 3), seed=516)
    arr49 = argus.GwbArray(big)
    with pytest.raises(Exception, match="48 pulsars"):
        argus.argus_gwb_loglik_grad(arr49, torch.from_numpy(thetas(49, 1, np.random.default_rng(1))).cuda())


def test_out_of_domain_and_host_pointers(argus):
    data = inputs.make_array(np.array([30, 40]), seed=504)
    theta = thetas(2, 5, np.random.default_rng(5))
    theta[0, 4] = 0.0           # EFAC of pulsar 0
    theta[1, 0] = np.inf
    arr = argus.GwbArray(data)
    ll_dev = run(argus, arr, theta)
    ll_host = argus.argus_gwb_loglik(arr, theta)        # numpy in, numpy out (staged)
    assert np.array_equal(ll_dev, ll_host)
    assert np.all(np.isneginf(ll_dev[:2])) and np.all(np.isfinite(ll_dev[2:]))
    assert ll_err(ll_dev, gwb.loglik(data, theta)) <= LL_TOL


def test_batch_larger_than_the_grid(argus):
    """More parameter vectors than resident blocks: the grid-stride loop."""
    data = inputs.make_array(np.array([12, 9]), seed=505)
    theta = thetas(2, 3000, np.random.default_rng(6))
    arr = argus.GwbArray(data)
    ll = run(argus, arr, theta)
    idx = np.array([0, 1, 1215, 1216, 2999])
    assert ll_err(ll[idx], gwb.loglik(data, theta[idx])) <= LL_TOL


G_TOL = 1e-6


def g_err(g, ref):
    g, ref = np.atleast_2d(g), np.atleast_2d(ref)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=1, keepdims=True))
    return np.nan_to_num(np.abs(g - ref) / scale, nan=np.inf).max()


@pytest.mark.parametrize("sizes", [[40], [30, 50, 20], [0, 25, 1, 60], [15] * 8])
def test_gradient_parity_small_arrays(argus, sizes):
    data = inputs.make_array(np.array(sizes), seed=510 + len(sizes), equad=1e-8)
    theta = thetas(len(sizes), 5, np.random.default_rng(10 + len(sizes)), lh=(-19.5, -18.3))
    arr = argus.GwbArray(data)
    th = torch.from_numpy(theta).cuda()
    ll, g = argus.argus_gwb_loglik_grad(arr, th)
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    ll_ref, g_ref = gwb.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL
    assert ll_err(ll, run(argus, arr, theta)) <= 1e-13
    assert g_err(g, g_ref) <= G_TOL


def test_gradient_with_equal_times(argus):
    data = inputs.make_array(np.array([40, 35, 25]), seed=511)
    a, b = data.off[1], data.off[2]
    data.t[a:a + 10] = data.t[3:13]
    data.t[a:b] = np.sort(data.t[a:b])
    data.t[b + 2:b + 5] = data.t[b + 2]
    theta = thetas(3, 4, np.random.default_rng(12), lh=(-19.5, -18.3))
    arr = argus.GwbArray(data)
    ll, g = argus.argus_gwb_loglik_grad(arr, torch.from_numpy(theta).cuda())
    ll_ref, g_ref = gwb.loglik_grad(data, theta)
    assert ll_err(ll.cpu().numpy(), ll_ref) <= LL_TOL
    assert g_err(g.cpu().numpy(), g_ref) <= G_TOL


def test_gradient_twenty_pulsars_vs_gpu_finite_differences(argus):
    """20 pulsars: Richardson central differences of the GPU likelihood."""
    data = inputs.make_array(np.full(20, 60), seed=512, equad=1e-8)
    th0 = thetas(20, 1, np.random.default_rng(13), lh=(-19.0, -18.6))[0]
    arr = argus.GwbArray(data)
    _, g = argus.argus_gwb_loglik_grad(arr, torch.from_numpy(th0[None, :]).cuda())
    g = g.cpu().numpy()[0]
    D = len(th0)
    rows = []
    for j in range(D):
        for h in (1e-4, 5e-5):
            for sgn in (1, -1):
                x = th0.copy(); x[j] += sgn * h
                rows.append(x)
    ll = run(argus, arr, np.array(rows))
    fd = np.array([(4 * (ll[4 * j + 2] - ll[4 * j + 3]) / 1e-4 - (ll[4 * j] - ll[4 * j + 1]) / 2e-4) / 3
                   for j in range(D)])
    assert g_err(g, fd) <= 1e-5


def test_gradient_out_of_domain_and_host_pointers(argus):
    data = inputs.make_array(np.array([30, 40]), seed=513)
    theta = thetas(2, 4, np.random.default_rng(14))
    theta[0, 4] = -1.0
    arr = argus.GwbArray(data)
    ll_h, g_h = argus.argus_gwb_loglik_grad(arr, theta)         # numpy (staged)
    ll_d, g_d = argus.argus_gwb_loglik_grad(arr, torch.from_numpy(theta).cuda())
    assert np.array_equal(ll_h, ll_d.cpu().numpy()) and np.array_equal(g_h, g_d.cpu().numpy())
    assert np.isneginf(ll_h[0]) and np.all(g_h[0] == 0.0)
    ll_ref, g_ref = gwb.loglik_grad(data, theta[1:])
    assert ll_err(ll_h[1:], ll_ref) <= LL_TOL and g_err(g_h[1:], g_ref) <= G_TOL


@pytest.mark.parametrize("lg_p,lg_a", [(-5.0, -8.0), (-8.0, -5.0), (-3.0, -3.0), (-5.5, -9.9)])
def test_fast_decays_fold_the_scaled_frame(argus, lg_p, lg_a):
    """Decay rates whose products over the TOA gaps fall below 2^-200 (and,
    at 1e-3 / s, to zero in a single gap): the likelihood kernel folds its
    scale factors back into the covariance and takes those predicts
    unscaled; the gradient kernel's checkpoint pass does the same."""
    data = inputs.make_array(np.array([40, 30, 25]), seed=514, equad=1e-8)
    theta = thetas(3, 4, np.random.default_rng(15), lh=(-19.5, -18.3))
    theta[:, 1] = lg_a
    theta[:, 3::3] = lg_p
    theta[1, 3] = -8.5                      # one pulsar slow: scales fold independently
    arr = argus.GwbArray(data)
    ll = run(argus, arr, theta)
    ll_ref, g_ref = gwb.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL
    ll_g, g = argus.argus_gwb_loglik_grad(arr, torch.from_numpy(theta).cuda())
    assert ll_err(ll_g.cpu().numpy(), ll_ref) <= LL_TOL
    assert g_err(g.cpu().numpy(), g_ref) <= G_TOL
