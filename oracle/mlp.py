"""Oracle of the surrogate network (TEST INFRASTRUCTURE ONLY).

The target path pairs the exact filter with a small learned surrogate of the
array log-likelihood and its gradient: an MLP 47 -> 4 x 256 (GELU) -> 48 with
BF16 weights and activations and FP32 accumulation, trained on the exact
filter's own evaluations and used as the first stage of delayed-acceptance
HMC.  This module is the plain numpy statement of what the GPU kernels
compute, with the same rounding points:

* layer l:  z_l = fp32( bf16(x_l) @ bf16(W_l)^T ) + b_l ;  x_{l+1} = bf16(gelu(z_l))
  for the four hidden layers, and y = fp32(bf16(x_4) @ bf16(W_4)^T) + b_4;
* gelu(z) = z/2 (1 + erf(z / sqrt 2)) (exact form), gelu'(z) = Phi(z) + z phi(z);
* loss L = sum_r sum_j w_j (y_rj - t_rj)^2 / n, dY = bf16(2 w_j (y - t) / n);
* backward: dW_l = fp32(dZ_l^T @ x_l), db_l = sum_r dZ_l (FP32 dZ),
  dX_l = fp32(bf16(dZ_l) @ bf16(W_l)),  dZ_{l-1} = dX_l * gelu'(z_{l-1});
* Adam with FP32 master weights (Kingma & Ba 2015), then BF16 copies.

Shapes are padded: input 47 -> 64 columns, output 48 -> 64 rows of W_4 (the
padding weights are zero and receive zero gradient).  With round=False every
BF16 rounding is skipped and the arithmetic runs in float64 -- the mode the
finite-difference pins use.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN_DIM, IN_PAD = 47, 64
OUT_DIM, OUT_PAD = 48, 64
HIDDEN = 256
LAYERS = [(IN_PAD, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, OUT_PAD)]


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int, in_dim: int = IN_DIM, out_dim: int = OUT_DIM):
    """Fan-in scaled normal weights, zero biases; padding entries zero."""
    rng = np.random.default_rng(seed)
    params = []
    for l, (k, n) in enumerate(LAYERS):
        fan_in = in_dim if l == 0 else k
        W = (rng.standard_normal((n, k)) * math.sqrt(2.0 / fan_in)).astype(np.float32)
        if l == 0:
            W[:, in_dim:] = 0.0
        if l == len(LAYERS) - 1:
            W = W * np.float32(0.5)
            W[out_dim:, :] = 0.0
        params.append([W, np.zeros(n, dtype=np.float32)])
    return params


def _r(x, rnd):
    return bf16_round(x) if rnd else x


def forward(params, x, rnd: bool = True):
    """x: [n, 64] standardized inputs.  Returns (y [n, 64], cache)."""
    dt = np.float32 if rnd else np.float64
    h = _r(np.asarray(x, dtype=dt), rnd)
    xs, zs = [], []
    for l, (W, b) in enumerate(params):
        xs.append(h)
        z = (h @ _r(W.astype(dt), rnd).T).astype(dt) + b.astype(dt)
        zs.append(z)
        if l < len(params) - 1:
            h = _r(gelu(z).astype(dt), rnd)
    return zs[-1], (xs, zs)


def loss_and_dy(y, t, w, rnd: bool = True):
    """Weighted MSE over the first OUT_DIM outputs; dY padded to OUT_PAD columns."""
    n = y.shape[0]
    d = y[:, :OUT_DIM] - t
    loss = float(np.sum(w[None, :] * d * d) / n)
    dy = np.zeros_like(y)
    dy[:, :OUT_DIM] = 2.0 * w[None, :] * d / n
    return loss, _r(dy.astype(y.dtype), rnd)


def backward(params, cache, dy, rnd: bool = True, return_dz: bool = False):
    """Gradients [(dW_l, db_l)] of the loss for dY = dL/dy (already rounded).
    return_dz: also return, per layer l, the rounded dL/dz_l it multiplied
    (dY for l = 4) and the FP32 dL/dz_l it summed for db_l."""
    xs, zs = cache
    dt = dy.dtype
    grads = [None] * len(params)
    dzs, dz32s = [None] * len(params), [None] * len(params)
    dz = dy
    dz_bf = dy
    for l in reversed(range(len(params))):
        W, _ = params[l]
        dzs[l], dz32s[l] = dz_bf, dz
        dW = (dz_bf.T @ xs[l]).astype(dt)
        db = dz.sum(axis=0).astype(dt)
        grads[l] = (dW, db)
        if l > 0:
            dx = (dz_bf @ _r(W.astype(dt), rnd)).astype(dt)
            dz = (dx * gelu_grad(zs[l - 1])).astype(dt)
            dz_bf = _r(dz, rnd)
    return (grads, dzs, dz32s) if return_dz else grads


def value_input_grad(params, x, rnd: bool = True, return_dz: bool = False):
    """d y_0 / d x: the value output's gradient with respect to the (standardized,
    padded) input, by back-propagating dY = e_0 with the same rounding points as
    the weight gradients (BF16 operands, FP32 accumulation).  return_dz: also
    return the rounded dy_0/dz_l of each layer l = 0..3 (index l)."""
    y, (xs, zs) = forward(params, x, rnd)
    dt = y.dtype
    dz_bf = np.zeros_like(y)
    dz_bf[:, 0] = 1.0
    dzs = [None] * len(params)
    for l in reversed(range(len(params))):
        W, _ = params[l]
        dx = (dz_bf @ _r(W.astype(dt), rnd)).astype(dt)
        if l == 0:
            return (y, dx, dzs) if return_dz else (y, dx)
        dz_bf = _r((dx * gelu_grad(zs[l - 1])).astype(dt), rnd)
        dzs[l - 1] = dz_bf


class Adam:
    """Adam on FP32 master weights (Kingma & Ba 2015), bias-corrected."""

    def __init__(self, params, beta1=0.9, beta2=0.999, eps=1e-8):
        self.b1, self.b2, self.eps = beta1, beta2, eps
        self.t = 0
        self.m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]

    def step(self, params, grads, lr):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for l, (gW, gb) in enumerate(grads):
            for i, g in enumerate((gW, gb)):
                g = g.astype(np.float32)
                m = self.m[l][i] = (self.b1 * self.m[l][i] + (1 - self.b1) * g).astype(np.float32)
                v = self.v[l][i] = (self.b2 * self.v[l][i] + (1 - self.b2) * g * g).astype(np.float32)
                upd = lr * (m / c1) / (np.sqrt(v / c2) + self.eps)
                params[l][i] = (params[l][i] - upd).astype(np.float32)
        return params


def train_step(params, opt, x, t, w, lr):
    y, cache = forward(params, x)
    loss, dy = loss_and_dy(y, t, w)
    grads = backward(params, cache, dy)
    opt.step(params, grads, lr)
    return loss, grads
