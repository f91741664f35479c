"""The boundary's remaining entry points on the GPU: per-walker status
(argus_walker_flags, ARGUS_ERR_NONFINITE on a synchronous call), and the
surrogate created for an array (argus_surrogate_create with and without a
weights file, argus_surrogate_save) and trained on packed exact outputs
(argus_surrogate_train_step)."""
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


def _theta_with_failures(data, B, seed):
    theta = inputs.make_theta_batch(data, B, seed=seed)
    theta[1, 8] = -1.0       # EFAC < 0: out of the domain
    theta[2, 3] = 1.5        # |cos iota| > 1: out of the domain
    theta[3, 7] = 200.0      # log10 sigma = 200: in the domain, sigma^2 overflows -> S = inf
    theta[5, 9] = 400.0      # the same on the second pulsar
    return theta


def test_walker_flags_tell_domain_from_filter_failure(argus):
    data = inputs.make_array(np.array([40, 70, 0, 15]), seed=401)
    theta = _theta_with_failures(data, 9, 402)
    arr = argus.argus_array_create(data)
    th = torch.from_numpy(theta).cuda()
    ll, g = argus.argus_loglik_grad(arr, th)        # device pointers: status OK
    flags = argus.argus_walker_flags(arr, th, ll)
    torch.cuda.synchronize()
    assert flags.cpu().numpy().tolist() == [0, 1, 1, 2, 0, 2, 0, 0, 0]
    ll = ll.cpu().numpy()
    assert np.all(np.isneginf(ll[[1, 2, 3, 5]])) and np.all(np.isfinite(ll[[0, 4, 6, 7, 8]]))
    assert np.all(g.cpu().numpy()[[1, 2, 3, 5]] == 0.0)
    good = [0, 4, 6, 7, 8]
    ll_ref = kalman.loglik(data, theta[good])
    assert np.max(np.abs(ll[good] - ll_ref) / np.maximum(np.abs(ll_ref), 1.0)) <= 1e-9


def test_host_call_reports_nonfinite_after_writing_every_output(argus):
    data = inputs.make_array(np.array([40, 70, 0, 15]), seed=401)
    theta = _theta_with_failures(data, 9, 402)
    arr = argus.argus_array_create(data)
    ll_d, g_d = argus.argus_loglik_grad(arr, torch.from_numpy(theta).cuda())
    ll_h = np.full(9, np.nan)
    g_h = np.full((9, data.dim), np.nan)
    with pytest.raises(argus.ArgusError) as e:
        argus.argus_loglik_grad(arr, theta, ll_h, g_h, strict=True)
    assert e.value.status == 4
    assert np.array_equal(ll_h, ll_d.cpu().numpy()) and np.array_equal(g_h, g_d.cpu().numpy())
    ll2 = argus.argus_loglik(arr, theta)             # default: -inf returned, no raise
    assert np.array_equal(ll2, ll_h)
    # out-of-domain walkers alone are ordinary rejections: status OK
    ok = theta[[0, 1, 2, 4]]
    argus.argus_loglik(arr, ok, strict=True)


def _array20(argus, seed=410):
    w = inputs.WORKLOADS["psr20_toa500-2000_w4096"]
    data = inputs.make_workload_array(w.name)
    return data, argus.argus_array_create(data)


def test_surrogate_create_for_array_and_weights_file(argus, tmp_path):
    from paper_2510_11077_gb300 import surrogate
    data, arr = _array20(argus)
    net = surrogate.Surrogate.from_array(arr)
    rng = np.random.default_rng(3)
    net.set_normalizers(rng.uniform(-1, 1, 47), rng.uniform(0.5, 2, 47), -123.0, 7.0, 3.0, 0.5)
    A = rng.standard_normal((47, 47)).astype(np.float32) / 47
    net.set_baseline(A @ A.T + 0.1 * np.eye(47, dtype=np.float32))
    x = torch.from_numpy(rng.standard_normal((300, 47)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal((300, 48)).astype(np.float32)).cuda()
    net.train_step_packed(x, y, 1e-3)
    path = tmp_path / "net.bin"
    net.save(path)
    assert path.stat().st_size == 8 + 16 + 4 * (surrogate.param_count() + 2 * 47 + 4 + 47 * 47)
    net2 = surrogate.Surrogate.from_array(arr, path)
    assert np.array_equal(net2.get_weights(), net.get_weights())
    for gm in (0, 1):
        net.set_grad_mode(gm)
        net2.set_grad_mode(gm)
        a, b = net.eval(x), net2.eval(x)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # a foreign or truncated file, and an array of another dimension, are refused
    bad = tmp_path / "bad.bin"
    bad.write_bytes(path.read_bytes()[:1000])
    with pytest.raises(surrogate.SurrogateError):
        surrogate.Surrogate.from_array(arr, bad)
    bad.write_bytes(b"NOTARGUS" + path.read_bytes()[8:])
    with pytest.raises(surrogate.SurrogateError):
        surrogate.Surrogate.from_array(arr, bad)
    other = argus.argus_array_create(inputs.make_array(np.array([30, 40]), seed=1))
    with pytest.raises(surrogate.SurrogateError, match="UNSUPPORTED"):
        surrogate.Surrogate.from_array(other)


def test_packed_train_step_equals_separate_targets(argus):
    """argus_surrogate_train_step on y = (loglik, gradient) rows gives the same
    step, bit for bit, as argus_surrogate_train_step_ex on the separate arrays."""
    from paper_2510_11077_gb300 import surrogate
    data, arr = _array20(argus)
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal((700, 47)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal((700, 48)).astype(np.float32)).cuda()
    nets = [surrogate.Surrogate.from_array(arr) for _ in range(2)]
    for n in nets:
        n.set_normalizers(np.zeros(47), np.ones(47), 0.1, 2.0, 2.0, 1.0)
    losses = []
    for _ in range(3):
        nets[0].train_step_packed(x, y, 1e-3)
        losses.append(nets[0].last_loss())
        l1 = nets[1].train_step(x, y[:, 0].contiguous(), y[:, 1:].contiguous(), 1e-3)
        assert losses[-1] == float(l1.item())
    assert np.array_equal(nets[0].get_weights(), nets[1].get_weights())
    assert losses[2] < losses[0]
