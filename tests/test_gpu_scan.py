"""GPU parity of the time-parallel (associative-scan) filter, plan mode
ARGUS_MODE_SCAN, against the CPU oracle and against the sequential filter.
Log-likelihood tolerance as everywhere: |d| <= 1e-9 max(|ll|, 1)."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from oracle import kalman
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


def run_ll(argus, arr, theta):
    return argus.argus_loglik(arr, torch.from_numpy(np.ascontiguousarray(theta)).cuda()).cpu().numpy()


def test_single_pulsar_1000_toas_one_walker(argus):
    """The few-lane workload the scan is for: 1 pulsar, 1000 TOAs, 1 walker."""
    w = inputs.WORKLOADS["psr1_toa1000"]
    data = inputs.make_workload_array(w.name)
    theta = inputs.make_theta_batch(data, 1, seed=w.seed)
    arr = argus.argus_array_create(data)
    ll_seq = run_ll(argus, arr, theta)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN)
    ll = run_ll(argus, arr, theta)
    assert ll_err(ll, kalman.loglik(data, theta)) <= LL_TOL
    assert ll_err(ll, ll_seq) <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 95, 1000, 4099])
@pytest.mark.parametrize("elems", [0, 1, 3])
def test_chunk_edges(argus, n, elems):
    data = inputs.make_array(np.array([n]), seed=400 + n, equad=1e-8)
    theta = inputs.make_theta_batch(data, 2, seed=1)
    arr = argus.argus_array_create(data)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN, scan_elems=elems)
    assert ll_err(run_ll(argus, arr, theta), kalman.loglik(data, theta)) <= LL_TOL


@pytest.mark.parametrize("model,pt", [("rw", False), ("ou", False), ("rw", True), ("ou", True)])
def test_ragged_array_all_models(argus, model, pt):
    data = inputs.make_array(np.array([0, 1, 37, 200, 513, 1290]), seed=401, equad=2e-8,
                             model=model, pulsar_term=pt)
    for kind in ("posterior", "prior"):
        theta = inputs.make_theta_batch(data, 5, seed=3, kind=kind)
        arr = argus.argus_array_create(data)
        arr.set_plan(mode=argus.ARGUS_MODE_SCAN)
        ll = run_ll(argus, arr, theta)
        assert ll_err(ll, kalman.loglik(data, theta)) <= LL_TOL
        lane = argus.argus_lane_loglik(arr, torch.from_numpy(theta).cuda()).cpu().numpy()
        _, ref = kalman.loglik(data, theta, lanes=True)
        assert ll_err(lane.ravel(), ref.ravel()) <= LL_TOL
        assert np.all(lane[:, 0] == 0.0)                   # the empty pulsar


def test_long_pulsar_and_equal_times(argus):
    data = inputs.make_array(np.array([20000, 3]), seed=402, model="ou")
    a = data.off[0]
    data.t[a + 100:a + 104] = data.t[a + 100]              # dt = 0 inside a chunk
    data.t[a + 63:a + 66] = data.t[a + 63]                 # ... and across a chunk edge
    data.t[a:data.off[1]] = np.sort(data.t[a:data.off[1]])
    theta = inputs.make_theta_batch(data, 1, seed=4)
    arr = argus.argus_array_create(data)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN, scan_elems=2)
    assert ll_err(run_ll(argus, arr, theta), kalman.loglik(data, theta)) <= LL_TOL


def test_out_of_domain_and_graph_replay(argus):
    data = inputs.make_array(np.array([300, 700]), seed=403)
    theta = inputs.make_theta_batch(data, 4, seed=5)
    theta[1, 8] = -1.0                                     # EFAC < 0
    theta[2, 0] = np.nan
    arr = argus.argus_array_create(data)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN)
    th = torch.from_numpy(theta).cuda()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    argus.argus_loglik(arr, th, out)                       # capture
    first = out.cpu().numpy().copy()
    for _ in range(3):
        argus.argus_loglik(arr, th, out)                   # replay
        assert np.array_equal(out.cpu().numpy(), first)
    assert np.all(np.isneginf(first[1:3])) and np.all(np.isfinite(first[[0, 3]]))
    assert ll_err(first, kalman.loglik(data, theta)) <= LL_TOL


# Gradient in plan mode SCAN: the time-parallel adjoint (suffix scan of the
# reverse sweep's affine maps, then each thread's own adjoint steps).  Against
# the oracle's complex-step gradient with the tolerance of every gradient
# test, |d| <= 1e-6 max(|g|, 1e-3 max|g|) per walker, and against the
# sequential adjoint (K3), which takes the same steps in another order.
G_TOL = 1e-6
G_SEQ_TOL = 1e-8


def g_err(g, ref):
    g, ref = np.atleast_2d(g), np.atleast_2d(ref)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=1, keepdims=True))
    scale = np.where(scale == 0, 1.0, scale)
    return np.nan_to_num(np.abs(g - ref) / scale, nan=np.inf).max()


def run_grad(argus, arr, theta):
    ll, g = argus.argus_loglik_grad(arr, torch.from_numpy(np.ascontiguousarray(theta)).cuda())
    torch.cuda.synchronize()
    return ll.cpu().numpy(), g.cpu().numpy()


def scan_and_sequential(argus, data, theta, elems=0):
    arr = argus.argus_array_create(data)
    seq = run_grad(argus, arr, theta)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN, scan_elems=elems)
    return run_grad(argus, arr, theta), seq


def test_gradient_single_pulsar_1000_toas_one_walker(argus):
    w = inputs.WORKLOADS["psr1_toa1000"]
    data = inputs.make_workload_array(w.name)
    theta = inputs.make_theta_batch(data, 1, seed=w.seed)
    (ll, g), (ll_s, g_s) = scan_and_sequential(argus, data, theta)
    ll_ref, g_ref = kalman.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL and g_err(g, g_ref) <= G_TOL
    assert ll_err(ll, ll_s) <= 1e-12 and g_err(g, g_s) <= G_SEQ_TOL


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 95, 1000, 4099])
@pytest.mark.parametrize("elems", [0, 1, 3])
def test_gradient_chunk_edges(argus, n, elems):
    data = inputs.make_array(np.array([n]), seed=410 + n, equad=1e-8)
    theta = inputs.make_theta_batch(data, 2, seed=2)
    (ll, g), (_, g_s) = scan_and_sequential(argus, data, theta, elems)
    ll_ref, g_ref = kalman.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL
    assert g_err(g, g_ref) <= G_TOL and g_err(g, g_s) <= G_SEQ_TOL


@pytest.mark.parametrize("model,pt", [("rw", False), ("ou", False), ("rw", True), ("ou", True)])
def test_gradient_ragged_array_all_models(argus, model, pt):
    data = inputs.make_array(np.array([0, 1, 37, 200, 513, 1290]), seed=411, equad=2e-8,
                             model=model, pulsar_term=pt)
    theta = inputs.make_theta_batch(data, 3, seed=7)
    (ll, g), (_, g_s) = scan_and_sequential(argus, data, theta)
    ll_ref, g_ref = kalman.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL
    assert g_err(g, g_ref) <= G_TOL and g_err(g, g_s) <= G_SEQ_TOL
    q = (data.dim - 7) // data.n_pulsars                  # parameters per pulsar
    assert np.all(g[:, 7:7 + q] == 0.0)                     # the empty pulsar


def test_gradient_long_pulsar_and_equal_times(argus):
    data = inputs.make_array(np.array([20000, 3]), seed=412, model="ou")
    a = data.off[0]
    data.t[a + 100:a + 104] = data.t[a + 100]              # dt = 0 inside a chunk
    data.t[a + 63:a + 66] = data.t[a + 63]                 # ... and across a chunk edge
    data.t[a:data.off[1]] = np.sort(data.t[a:data.off[1]])
    theta = inputs.make_theta_batch(data, 1, seed=8)
    (ll, g), (_, g_s) = scan_and_sequential(argus, data, theta, elems=2)
    ll_ref, g_ref = kalman.loglik_grad(data, theta)
    assert ll_err(ll, ll_ref) <= LL_TOL
    assert g_err(g, g_ref) <= G_TOL and g_err(g, g_s) <= G_SEQ_TOL


def test_gradient_every_lane_empty(argus):
    full = inputs.make_array(np.array([1, 1]), seed=413)
    theta = inputs.make_theta_batch(full, 2, seed=9)
    none = np.empty(0)
    data = dataclasses.replace(full, off=np.zeros(3, dtype=np.int64), t=none, r=none, sigma=none)
    ll_ref, g_ref = kalman.loglik_grad(data, theta)
    assert np.all(ll_ref == 0.0) and np.all(g_ref == 0.0)
    arr = argus.argus_array_create(data)
    for plan in (dict(mode=argus.ARGUS_MODE_BATCHED), dict(mode=argus.ARGUS_MODE_SCAN)):
        arr.set_plan(**plan)
        ll, g = run_grad(argus, arr, theta)
        assert np.all(ll == 0.0) and np.all(g == 0.0)
        assert np.all(run_ll(argus, arr, theta) == 0.0)


def test_gradient_out_of_domain_replay_host_buffers_and_determinism(argus):
    data = inputs.make_array(np.array([300, 700]), seed=414)
    theta = inputs.make_theta_batch(data, 4, seed=10)
    theta[1, 8] = -1.0                                     # EFAC < 0
    theta[2, 0] = np.nan
    arr = argus.argus_array_create(data)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN)
    th = torch.from_numpy(theta).cuda()
    ll = torch.empty(4, dtype=torch.float64, device="cuda")
    g = torch.empty((4, data.dim), dtype=torch.float64, device="cuda")
    argus.argus_loglik_grad(arr, th, ll, g)                # capture
    first = (ll.cpu().numpy().copy(), g.cpu().numpy().copy())
    for _ in range(3):
        argus.argus_loglik_grad(arr, th, ll, g)            # replay
        assert np.array_equal(ll.cpu().numpy(), first[0]) and np.array_equal(g.cpu().numpy(), first[1])
    assert np.all(np.isneginf(first[0][1:3])) and np.all(first[1][1:3] == 0.0)
    ll_h, g_h = argus.argus_loglik_grad(arr, theta)        # host buffers, staged copies
    assert np.array_equal(np.asarray(ll_h), first[0]) and np.array_equal(np.asarray(g_h), first[1])
    ok = [0, 3]
    ll_ref, g_ref = kalman.loglik_grad(data, theta[ok])
    assert ll_err(first[0][ok], ll_ref) <= LL_TOL and g_err(first[1][ok], g_ref) <= G_TOL
    ll2 = argus.argus_loglik(arr, th).cpu().numpy()        # the loglik-only path of the same plan
    assert ll_err(ll2, first[0]) <= 1e-12


def test_large_batch_chunking_loglik_and_gradient(argus):
    """1024 walkers on one 1000-TOA pulsar: the automatic chunking is capped
    at the pulsar's TOAs / 32 per thread (one full chunk per lane); the scan
    still agrees with the batched filter and its adjoint."""
    data = inputs.make_array(np.array([1000]), seed=415)
    theta = inputs.make_theta_batch(data, 1024, seed=11)
    (ll, g), (ll_s, g_s) = scan_and_sequential(argus, data, theta)
    assert ll_err(ll, ll_s) <= 1e-12 and g_err(g, g_s) <= G_SEQ_TOL
    ll_ref, g_ref = kalman.loglik_grad(data, theta[:4])
    assert ll_err(ll[:4], ll_ref) <= LL_TOL and g_err(g[:4], g_ref) <= G_TOL
    arr = argus.argus_array_create(data)
    arr.set_plan(mode=argus.ARGUS_MODE_SCAN)
    assert ll_err(run_ll(argus, arr, theta), ll_s) <= 1e-12
