"""Pins of the surrogate-network oracle (oracle/mlp.py) against facts outside it:
torch's own BF16 conversion, the erf closed form of GELU, finite differences
of the loss, explicit loops on a tiny batch, and Adam's closed-form steps."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10 ** rng.uniform(-8, 8, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.001953125, 3e38, 1e-40], np.float32)])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_gelu_closed_form_and_derivative():
    z = np.linspace(-6, 6, 121)
    ref = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    assert np.allclose(mlp.gelu(z), ref, rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)
    # textbook values: gelu(0) = 0, gelu'(0) = 1/2, gelu(z) -> z for large z
    assert mlp.gelu(np.array([0.0]))[0] == 0.0 and mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-20


def _tiny_params(seed):
    p = mlp.init_params(seed)
    return [[W.astype(np.float64), b.astype(np.float64) + 0.01 * (l + 1)] for l, (W, b) in enumerate(p)]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = _tiny_params(3)
    x = np.zeros((6, mlp.IN_PAD)); x[:, :mlp.IN_DIM] = rng.standard_normal((6, mlp.IN_DIM))
    t = rng.standard_normal((6, mlp.OUT_DIM))
    w = np.concatenate([[4.0], np.ones(mlp.OUT_DIM - 1)])

    def loss(ps):
        y, _ = mlp.forward(ps, x, rnd=False)
        return mlp.loss_and_dy(y, t, w, rnd=False)[0]

    y, cache = mlp.forward(params, x, rnd=False)
    _, dy = mlp.loss_and_dy(y, t, w, rnd=False)
    grads = mlp.backward(params, cache, dy, rnd=False)
    h = 1e-6
    for l in range(len(params)):
        for which in (0, 1):
            arr = params[l][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, 5, replace=False):
                if which == 0 and l == 0 and (idx % mlp.IN_PAD) >= mlp.IN_DIM:
                    continue
                old = flat[idx]
                flat[idx] = old + h; lp = loss(params)
                flat[idx] = old - h; lm = loss(params)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[l][which].reshape(-1)[idx]
                # central differences at h = 1e-6 carry ~1e-9 absolute roundoff (loss ~ 10)
                assert abs(an - fd) <= 1e-5 * max(abs(fd), 1e-3), (l, which, idx, an, fd)


def test_forward_matches_explicit_loops():
    rng = np.random.default_rng(2)
    params = mlp.init_params(5)
    x = np.zeros((2, mlp.IN_PAD), np.float32); x[:, :mlp.IN_DIM] = rng.standard_normal((2, mlp.IN_DIM))
    y, _ = mlp.forward(params, x, rnd=False)
    for r in range(2):
        h = [float(v) for v in x[r]]
        for l, (W, b) in enumerate(params):
            z = [sum(float(W[o, i]) * h[i] for i in range(len(h))) + float(b[o]) for o in range(W.shape[0])]
            h = [0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z] if l < 4 else z
        assert np.allclose(y[r], h, rtol=1e-10, atol=1e-12)


def test_bf16_forward_close_to_exact_forward():
    rng = np.random.default_rng(3)
    params = mlp.init_params(6)
    x = np.zeros((64, mlp.IN_PAD), np.float32); x[:, :mlp.IN_DIM] = rng.standard_normal((64, mlp.IN_DIM))
    y16, _ = mlp.forward(params, x, rnd=True)
    params64 = [[mlp.bf16_round(W).astype(np.float64), b.astype(np.float64)] for W, b in params]
    y64, _ = mlp.forward(params64, mlp.bf16_round(x).astype(np.float64), rnd=False)
    # BF16 activations: relative error of a few 2^-8 per layer
    assert np.max(np.abs(y16 - y64)) <= 0.05 * np.max(np.abs(y64))


def test_adam_closed_form_steps():
    params = [[np.array([[1.0]], np.float32), np.array([0.0], np.float32)]]
    opt = mlp.Adam(params)
    g = [(np.array([[0.3]], np.float32), np.array([-2.0], np.float32))]
    opt.step(params, g, lr=0.01)
    # first bias-corrected step is -lr * sign(g)
    assert params[0][0][0, 0] == pytest.approx(1.0 - 0.01, rel=1e-6)
    assert params[0][1][0] == pytest.approx(0.0 + 0.01, rel=1e-6)
    g2 = [(np.array([[0.1]], np.float32), np.array([-2.0], np.float32))]
    opt.step(params, g2, lr=0.01)
    m = 0.9 * 0.1 * 0.3 + 0.1 * 0.1
    v = 0.999 * 0.001 * 0.09 + 0.001 * 0.01
    step = 0.01 * (m / (1 - 0.81)) / (math.sqrt(v / (1 - 0.999 ** 2)) + 1e-8)
    assert params[0][0][0, 0] == pytest.approx(0.99 - step, rel=1e-6)


def test_training_reduces_loss_and_keeps_padding_zero():
    rng = np.random.default_rng(4)
    params = mlp.init_params(7)
    opt = mlp.Adam(params)
    n = 256
    x = np.zeros((n, mlp.IN_PAD), np.float32); x[:, :mlp.IN_DIM] = rng.standard_normal((n, mlp.IN_DIM))
    t = np.tanh(x[:, :mlp.OUT_DIM] * 0.5)
    w = np.ones(mlp.OUT_DIM, np.float32)
    losses = [mlp.train_step(params, opt, x, t, w, 3e-3)[0] for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0]
    assert np.all(params[0][0][:, mlp.IN_DIM:] == 0) and np.all(params[4][0][mlp.OUT_DIM:] == 0)
    assert np.all(params[4][1][mlp.OUT_DIM:] == 0)


def test_value_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(8)
    params = _tiny_params(9)
    x = np.zeros((3, mlp.IN_PAD)); x[:, :mlp.IN_DIM] = rng.standard_normal((3, mlp.IN_DIM))
    _, g = mlp.value_input_grad(params, x, rnd=False)
    h = 1e-6
    for k in rng.choice(mlp.IN_DIM, 8, replace=False):
        xp, xm = x.copy(), x.copy(); xp[:, k] += h; xm[:, k] -= h
        fd = (mlp.forward(params, xp, rnd=False)[0][:, 0] - mlp.forward(params, xm, rnd=False)[0][:, 0]) / (2 * h)
        assert np.allclose(g[:, k], fd, rtol=1e-5, atol=1e-7)
