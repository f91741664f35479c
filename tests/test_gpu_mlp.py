"""Surrogate network on the GPU against its oracle (oracle/mlp.py).

The BF16 rounding points match the oracle's; the remaining differences come
from FP32 summation order inside the tensor cores, which can move an
activation across a BF16 rounding boundary.  Tolerances below are stated
relative to the largest magnitude of each compared array.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2510_11077_gb300 import argus
    lib = argus.load()
    vp = ctypes.c_void_p
    lib.argus_selftest_gemm.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, vp]
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return lib


def _bf16_bits(x):
    r = mlp.bf16_round(x)
    return (r.view(np.uint32) >> 16).astype(np.uint16), r


@pytest.mark.parametrize("M,N,K,bn,chunks", [(128, 64, 64, 64, 1), (128, 128, 256, 128, 1),
                                             (256, 256, 256, 128, 1), (256, 64, 512, 64, 2),
                                             (384, 128, 256, 128, 2)])
def test_tensor_core_gemm(lib, M, N, K, bn, chunks):
    rng = np.random.default_rng(M + N + K)
    A16, A = _bf16_bits(rng.standard_normal((M, K)).astype(np.float32))
    B16, B = _bf16_bits(rng.standard_normal((N, K)).astype(np.float32))
    C = np.empty((chunks, M, N), np.float32)
    st = lib.argus_selftest_gemm(A16.ctypes.data, B16.ctypes.data, M, N, K, bn, chunks, C.ctypes.data)
    assert st == 0, st
    kc = K // chunks
    for z in range(chunks):
        ref = A[:, z * kc:(z + 1) * kc].astype(np.float64) @ B[:, z * kc:(z + 1) * kc].astype(np.float64).T
        assert np.max(np.abs(C[z] - ref)) <= 1e-5 * np.max(np.abs(ref)), z


def _oracle_io(params, theta, xm, xs, ym, ys):
    x = np.zeros((theta.shape[0], mlp.IN_PAD), np.float32)
    x[:, :mlp.IN_DIM] = (theta.astype(np.float32) - xm) / xs
    y, cache = mlp.forward(params, x)
    ll = y[:, 0] * np.float32(ys) + np.float32(ym)
    g = y[:, 1:mlp.OUT_DIM] * np.float32(ys) / xs
    return x, y, cache, ll, g


def _setup(seed, n):
    from paper_2510_11077_gb300 import surrogate
    rng = np.random.default_rng(seed)
    params = mlp.init_params(seed)
    for l in range(5):   # non-zero biases so the bias path is exercised
        params[l][1] = (0.1 * rng.standard_normal(params[l][1].shape)).astype(np.float32)
        if l == 4:
            params[l][1][mlp.OUT_DIM:] = 0.0
    theta = rng.uniform(-3, 3, (n, mlp.IN_DIM)).astype(np.float32)
    xm = rng.uniform(-0.5, 0.5, mlp.IN_DIM).astype(np.float32)
    xs = rng.uniform(0.5, 2.0, mlp.IN_DIM).astype(np.float32)
    ym, ys = 1234.5, 17.0
    s = surrogate.Surrogate(device=0, max_rows=1024, seed=seed)
    s.set_normalizers(xm, xs, ym, ys, value_weight=2.0, grad_weight=1.0)
    s.set_weights(surrogate.flatten(params))
    return s, params, theta, xm, xs, ym, ys


def test_surrogate_weights_roundtrip(lib):
    s, params, *_ = _setup(11, 8)
    from paper_2510_11077_gb300 import surrogate
    assert np.array_equal(s.get_weights(), surrogate.flatten(params))


@pytest.mark.parametrize("n", [1, 130, 1000, 2500])
def test_surrogate_eval_matches_oracle(lib, n):
    s, params, theta, xm, xs, ym, ys = _setup(12, n)
    ll, g = s.eval(torch.from_numpy(theta).cuda())
    s.check()
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    _, y, _, ll_ref, g_ref = _oracle_io(params, theta, xm, xs, ym, ys)
    dv = np.abs(ll - ll_ref) / ys
    assert dv.max() <= 2e-2 * max(np.abs(y[:, 0]).max(), 1e-3), dv.max()
    dg = np.abs(g - g_ref)
    assert dg.max() <= 2e-2 * np.abs(g_ref).max(), (dg.max(), np.abs(g_ref).max())
    # the bulk agrees far more tightly than the worst element
    assert np.median(dg) <= 1e-3 * np.abs(g_ref).max()


def test_surrogate_train_step_gradients_match_oracle(lib):
    from paper_2510_11077_gb300 import surrogate
    n = 512
    s, params, theta, xm, xs, ym, ys = _setup(13, n)
    rng = np.random.default_rng(5)
    ll_t = (ym + ys * rng.standard_normal(n)).astype(np.float32)
    g_t = (rng.standard_normal((n, mlp.IN_DIM)) * ys / xs).astype(np.float32)
    loss = s.train_step(torch.from_numpy(theta).cuda(), torch.from_numpy(ll_t).cuda(),
                        torch.from_numpy(g_t).cuda(), lr=1e-3)
    s.check()
    gpu = surrogate.unflatten(s.last_grads(), mlp.LAYERS)
    x, y, cache, _, _ = _oracle_io(params, theta, xm, xs, ym, ys)
    t = np.zeros((n, mlp.OUT_DIM), np.float32)
    t[:, 0] = (ll_t - np.float32(ym)) / np.float32(ys)
    t[:, 1:] = g_t * xs / np.float32(ys)
    w = np.concatenate([[2.0], np.ones(mlp.OUT_DIM - 1)]).astype(np.float32)
    loss_ref, dy = mlp.loss_and_dy(y, t, w)
    assert abs(float(loss.item()) - loss_ref) <= 1e-3 * loss_ref
    ref = mlp.backward(params, cache, dy)
    for l in range(5):
        for i in range(2):
            a, b = gpu[l][i], ref[l][i]
            assert np.max(np.abs(a - b)) <= 3e-2 * np.max(np.abs(b)), (l, i)
            cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))
            assert cos > 0.999, (l, i, cos)
    # padding stays zero after the Adam step
    wts = surrogate.unflatten(s.get_weights(), mlp.LAYERS)
    assert np.all(wts[0][0][:, mlp.IN_DIM:] == 0) and np.all(wts[4][0][mlp.OUT_DIM:] == 0)
    assert np.all(wts[4][1][mlp.OUT_DIM:] == 0)


def test_surrogate_training_fits_a_smooth_function(lib):
    """Adam on the GPU drives the loss of a smooth target well down (as the
    oracle does on the same problem)."""
    from paper_2510_11077_gb300 import surrogate
    rng = np.random.default_rng(7)
    n = 1024
    theta = rng.standard_normal((n, mlp.IN_DIM)).astype(np.float32)
    A = rng.standard_normal((mlp.IN_DIM, mlp.IN_DIM)).astype(np.float32) / mlp.IN_DIM
    ll = -0.5 * np.einsum("ni,ij,nj->n", theta, A @ A.T + np.eye(mlp.IN_DIM), theta).astype(np.float32)
    g = -(theta @ (A @ A.T + np.eye(mlp.IN_DIM))).astype(np.float32)
    s = surrogate.Surrogate(device=0, max_rows=1024, seed=3)
    s.set_normalizers(np.zeros(mlp.IN_DIM), np.ones(mlp.IN_DIM), float(ll.mean()), float(ll.std()))
    th, l_, g_ = (torch.from_numpy(a).cuda() for a in (theta, ll, g))
    losses = [float(s.train_step(th, l_, g_, lr=2e-3).item()) for _ in range(150)]
    s.check()
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])


def test_surrogate_value_backprop_gradient_matches_oracle(lib):
    n = 700
    s, params, theta, xm, xs, ym, ys = _setup(14, n)
    s.set_grad_mode(1)
    ll, g = s.eval(torch.from_numpy(theta).cuda())
    s.check()
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    x = np.zeros((n, mlp.IN_PAD), np.float32)
    x[:, :mlp.IN_DIM] = (theta.astype(np.float32) - xm) / xs
    y, dx = mlp.value_input_grad(params, x)
    g_ref = dx[:, :mlp.IN_DIM] * np.float32(ys) / xs
    assert np.max(np.abs(ll - (y[:, 0] * ys + ym))) <= 2e-2 * ys * max(np.abs(y[:, 0]).max(), 1e-3)
    dg = np.abs(g - g_ref)
    assert dg.max() <= 3e-2 * np.abs(g_ref).max(), (dg.max(), np.abs(g_ref).max())
    assert np.median(dg) <= 2e-3 * np.abs(g_ref).max()


@pytest.mark.parametrize("n", [1, 127, 130, 1000, 2500])
@pytest.mark.parametrize("mode", ["value", "gradient head", "value backprop"])
@pytest.mark.parametrize("baseline", [False, True])
def test_fused_eval_matches_layer_by_layer(lib, n, mode, baseline):
    """The fused kernel (all layers, and the value output's back-propagation,
    in one launch per 1024 rows) against the one-GEMM-per-layer path on the
    same weights and inputs.  Both take the same BF16 operands and the same
    FP32 accumulation order in the tensor cores, so they agree to the
    rounding of a few FP32 operations in the epilogues; the bound, 1e-4 of
    the largest magnitude, is far inside the 2e-2 both keep to the oracle."""
    s, params, theta, xm, xs, ym, ys = _setup(20 + n, n)
    if baseline:
        rng = np.random.default_rng(n)
        A = rng.standard_normal((mlp.IN_DIM, mlp.IN_DIM)).astype(np.float32) / mlp.IN_DIM
        s.set_baseline(A @ A.T + 0.1 * np.eye(mlp.IN_DIM, dtype=np.float32))
    if mode == "value backprop":
        s.set_grad_mode(1)
    with_grad = mode != "value"
    th = torch.from_numpy(theta).cuda()
    out = {}
    for fused in (False, True):
        s.set_fused(fused)
        r = s.eval(th, with_grad=with_grad)
        s.check()
        out[fused] = [x.cpu().numpy() for x in (r if with_grad else (r,))]
    for ref, got in zip(out[False], out[True]):
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), np.max(np.abs(got - ref))
    # a second call on the same handle gives the same result (the scratch is rewritten)
    r = s.eval(th, with_grad=with_grad)
    again = [x.cpu().numpy() for x in (r if with_grad else (r,))]
    for a_, b_ in zip(again, out[True]):
        assert np.array_equal(a_, b_)


@pytest.mark.parametrize("n", [1, 300, 2500])
@pytest.mark.parametrize("grad_mode", [0, 1])
def test_eval_f64_equals_eval_with_conversions(lib, n, grad_mode):
    """argus_surrogate_eval_f64 does the sampler's conversions inside the fused
    kernel: it must equal argus_surrogate_eval on float(z - centre) followed by
    the double conversion, the offset and the -inf of a non-finite value,
    bit for bit."""
    s, params, theta, xm, xs, ym, ys = _setup(40 + n, n)
    rng = np.random.default_rng(n)
    A = rng.standard_normal((mlp.IN_DIM, mlp.IN_DIM)).astype(np.float32) / mlp.IN_DIM
    s.set_baseline(A @ A.T + 0.1 * np.eye(mlp.IN_DIM, dtype=np.float32))
    s.set_grad_mode(grad_mode)
    centre = torch.from_numpy(rng.standard_normal(mlp.IN_DIM)).cuda()
    z = torch.from_numpy(theta.astype(np.float64) + rng.standard_normal(theta.shape) * 1e-3).cuda() + centre
    off = -1234.5678
    ll_f, g_f = s.eval((z - centre).float().contiguous())
    ref_ll = ll_f.double() + off
    ref_ll = torch.where(torch.isfinite(ref_ll), ref_ll, torch.full_like(ref_ll, -np.inf))
    for _ in range(2):
        ll, g = s.eval_z(z, centre, off)
        s.check()
        assert torch.equal(ll, ref_ll) and torch.equal(g, g_f.double())
    ll_only = s.eval_z(z, centre, off, with_grad=False)
    assert torch.equal(ll_only, ref_ll)
