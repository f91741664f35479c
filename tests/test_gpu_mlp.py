"""Surrogate network on the GPU against its oracle (oracle/mlp.py).

The BF16 rounding points match the oracle's; the remaining differences come
from FP32 summation order inside the tensor cores, which can move an
activation across a BF16 rounding boundary.  Every kernel is checked two
ways (bounds in tests/mlp_bounds.py): layer by layer, each GEMM on the GPU's
own BF16 operands, within the FP32 accumulation bound, and each BF16 epilogue
equal to the oracle's rounding except at a rounding boundary; and end to end,
the oracle run on its own, element by element within a bound carried through
the network's rounding points.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from oracle import mlp
from tests import mlp_bounds as B

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


MODES = {"value": (0, False), "gradient head": (0, True), "value backprop": (1, True)}


def _traced_eval(lib, s, theta, with_grad):
    """Fused evaluation with the stage trace on: outputs, and per GEMM stage
    its BF16 A operand and FP32 accumulator ([9][n][256] each)."""
    n = theta.shape[0]
    act = torch.zeros((9, n, 256), dtype=torch.float32, device="cuda")
    acc = torch.zeros((9, n, 256), dtype=torch.float32, device="cuda")
    vp = ctypes.c_void_p
    lib.argus_selftest_surrogate_trace.argtypes = [vp, vp, vp, ctypes.c_int64]
    assert lib.argus_selftest_surrogate_trace(s.handle, act.data_ptr(), acc.data_ptr(), n) == 0
    r = s.eval(torch.from_numpy(theta).cuda(), with_grad=with_grad)
    s.check()
    assert lib.argus_selftest_surrogate_trace(s.handle, None, None, 0) == 0
    out = [x.cpu().numpy() for x in (r if with_grad else (r,))]
    return out, act.cpu().numpy().astype(np.float64), acc.cpu().numpy()


def _f32_out_close(got, ref_terms, ref, what):
    """Outputs formed from a checked FP32 value by a few FP32 operations
    (de-standardization, offsets): within 4 FP32 roundings of their terms."""
    tol = 4.0 * B.U32 * ref_terms + 1e-30
    err = np.abs(np.asarray(got, np.float64) - ref)
    assert np.all(err <= tol), (what, float((err / tol).max()))


@pytest.mark.parametrize("n,cluster", [(1, 0), (130, 1), (130, 2), (130, 4), (1000, 0), (2500, 1),
                                       (2500, 4)])
@pytest.mark.parametrize("mode", list(MODES))
def test_fused_stages_match_oracle_layer_by_layer(lib, n, cluster, mode):
    """Each of the fused kernel's GEMM stages against the oracle's arithmetic
    on the GPU's own BF16 operands (so that no rounding flip can compound):
    every accumulator element within gamma_K of its absolute sum (1e-3 of its
    own scale), every BF16 activation equal to the oracle's rounding of the
    epilogue (GELU, gelu', products) except at a rounding boundary within the
    FP32 evaluation error, and the outputs within 4 FP32 roundings of the
    de-standardized accumulator."""
    grad_mode, with_grad = MODES[mode]
    s, params, theta, xm, xs, ym, ys = _setup(60 + n, n)
    s.set_grad_mode(grad_mode)
    s.set_cluster(cluster)
    out, act, acc = _traced_eval(lib, s, theta, with_grad)
    W16 = B.weights16(params)
    bias = [np.asarray(b, np.float32) for _, b in params]
    x = np.zeros((n, mlp.IN_PAD), np.float32)
    x[:, :mlp.IN_DIM] = (theta - xm) / xs
    # stage 0's operand is the standardized input, rounded to BF16
    assert np.array_equal(act[0][:, :mlp.IN_PAD], B.bf16_round64(x))
    z32 = []
    for st in range(5):
        K = mlp.IN_PAD if st == 0 else mlp.HIDDEN
        N = mlp.HIDDEN if st < 4 else mlp.OUT_DIM
        B.check_acc(acc[st][:, :N], act[st][:, :K], W16[st][:N], f"stage {st}")
        z = acc[st][:, :N] + bias[st][:N]                       # the FP32 bias add
        z32.append(z)
        if st < 4:
            zz = z.astype(np.float64)
            u = mlp.gelu(zz)
            B.check_rounded(act[st + 1][:, :mlp.HIDDEN], u, B.fn_err(zz, u) + B.U32 * np.abs(u),
                            f"h{st + 1}")
    y = z32[4].astype(np.float64)
    _f32_out_close(out[0], np.abs(y[:, 0] * ys) + abs(ym), y[:, 0] * ys + ym, "loglik")
    if mode == "gradient head":
        g_ref = y[:, 1:] * ys / xs.astype(np.float64)
        _f32_out_close(out[1], np.abs(g_ref), g_ref, "gradient outputs")
    if mode == "value backprop":
        # seed: W_4[0] * gelu'(z_3), then back through W_3, W_2, W_1 and W_0
        z3 = z32[3].astype(np.float64)
        gp = mlp.gelu_grad(z3)
        u = W16[4][0][None, :] * gp
        B.check_rounded(act[5][:, :mlp.HIDDEN], u,
                        np.abs(W16[4][0][None, :]) * B.fn_err(z3, gp) + B.U32 * np.abs(u), "dz3")
        for st in (5, 6, 7):
            l = 8 - st
            B.check_acc(acc[st][:, :mlp.HIDDEN], act[st][:, :mlp.HIDDEN], W16[l], f"stage {st}",
                        transposed=False)
            zz = z32[l - 1].astype(np.float64)
            gp = mlp.gelu_grad(zz)
            a = acc[st][:, :mlp.HIDDEN].astype(np.float64)
            u = a * gp
            B.check_rounded(act[st + 1][:, :mlp.HIDDEN], u,
                            np.abs(a) * B.fn_err(zz, gp) + B.U32 * np.abs(u), f"dz{l - 1}")
        B.check_acc(acc[8][:, :mlp.IN_DIM], act[8][:, :mlp.HIDDEN], W16[0][:, :mlp.IN_DIM],
                    "stage 8", transposed=False)
        g_ref = acc[8][:, :mlp.IN_DIM].astype(np.float64) * ys / xs.astype(np.float64)
        _f32_out_close(out[1], np.abs(g_ref), g_ref, "back-propagated gradient")


@pytest.mark.parametrize("n", [1, 130, 1000, 2500])
@pytest.mark.parametrize("mode", list(MODES))
def test_fused_eval_matches_oracle_within_derived_bound(lib, n, mode):
    """End to end: the fused kernel's outputs against the oracle run on its
    own (mlp.forward, mlp.value_input_grad), element by element.  The bound
    (tests/mlp_bounds.py) is the last rounding point's flips carried through
    the output layer's weights plus each side's FP32 accumulation bound, and
    4 FP32 roundings of the de-standardization; the flips at every rounding
    point (four for the forward pass, four more for the back-propagation)
    must stay below 1% of the values."""
    grad_mode, with_grad = MODES[mode]
    s, params, theta, xm, xs, ym, ys = _setup(80 + n, n)
    s.set_grad_mode(grad_mode)
    out, act, _ = _traced_eval(lib, s, theta, with_grad)
    out = [o.astype(np.float64) for o in out]
    x, y, (xs_o, zs_o), ll_o, g_o = _oracle_io(params, theta, xm, xs, ym, ys)
    W16 = B.weights16(params)
    xs64 = xs.astype(np.float64)
    d = [None] + [B.flips(act[l][:, :mlp.HIDDEN], xs_o[l], f"h{l}") for l in range(1, 5)]
    h4g, h4o = act[4][:, :mlp.HIDDEN], xs_o[4]
    by = B.last_layer_bound(d[4], h4g, h4o, W16[4][:mlp.OUT_DIM].T)
    by += 2.0 * B.U32 * np.abs(y[:, :mlp.OUT_DIM].astype(np.float64))       # each side's bias add
    checks = [(out[0], ll_o, by[:, 0] * ys, np.abs(y[:, 0] * ys) + abs(ym))]
    if mode == "gradient head":
        checks.append((out[1], g_o, by[:, 1:] * ys / xs64, np.abs(g_o)))
    if mode == "value backprop":
        _, dx_o, dz_o = mlp.value_input_grad(params, x, return_dz=True)
        dd = {l: B.flips(act[8 - l][:, :mlp.HIDDEN], dz_o[l], f"dz{l}") for l in range(4)}
        bx = B.last_layer_bound(dd[0], act[8][:, :mlp.HIDDEN], dz_o[0], W16[0][:, :mlp.IN_DIM])
        g_o = dx_o[:, :mlp.IN_DIM].astype(np.float64) * ys / xs64
        checks.append((out[1], g_o, bx * ys / xs64, np.abs(g_o)))
    for got, ref, T, terms in checks:
        ref = np.asarray(ref, np.float64)
        tol = T + 4.0 * B.U32 * terms + 1e-30
        err = np.abs(got - ref)
        assert np.all(err <= tol), (mode, float((err / tol).max()), int(np.sum(err > tol)))


def _train_setup(lib, seed, n):
    s, params, theta, xm, xs, ym, ys = _setup(seed, n)
    rng = np.random.default_rng(seed + 1)
    ll_t = (ym + ys * rng.standard_normal(n)).astype(np.float32)
    g_t = (rng.standard_normal((n, mlp.IN_DIM)) * ys / xs).astype(np.float32)
    lib.argus_selftest_surrogate_keep.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    assert lib.argus_selftest_surrogate_keep(s.handle, 1) == 0
    loss = s.train_step(torch.from_numpy(theta).cuda(), torch.from_numpy(ll_t).cuda(),
                        torch.from_numpy(g_t).cuda(), lr=1e-3)
    s.check()
    t = np.zeros((n, mlp.OUT_DIM), np.float32)
    t[:, 0] = (ll_t - np.float32(ym)) / np.float32(ys)
    t[:, 1:] = g_t * xs / np.float32(ys)
    w = np.concatenate([[2.0], np.ones(mlp.OUT_DIM - 1)]).astype(np.float32)
    return s, params, theta, xm, xs, ym, ys, t, w, float(loss.item())


def _buffer(lib, s, which, layer, shape, dtype):
    vp = ctypes.c_void_p
    lib.argus_selftest_surrogate_buffer.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp,
                                                    ctypes.c_int64]
    a = np.empty(shape, dtype)
    assert lib.argus_selftest_surrogate_buffer(s.handle, which, layer, a.ctypes.data, a.nbytes) == 0, \
        lib.argus_surrogate_last_error()
    if dtype == np.uint16:
        return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return a.astype(np.float64)


@pytest.mark.parametrize("n", [130, 512])
def test_surrogate_train_step_matches_oracle_layer_by_layer(lib, n):
    """A training step's every product against the oracle's arithmetic on the
    GPU's own operands: forward pre-activations and activations, the loss
    gradient dY, each back-propagated dZ (FP32, and its BF16 rounding), and
    the weight and bias gradients (split-K partials summed in fixed order)
    within the FP32 accumulation bound of their sums."""
    from paper_2510_11077_gb300 import surrogate
    s, params, theta, xm, xs, ym, ys, t, w, loss = _train_setup(lib, 13 + n, n)
    R = ((n + 127) // 128) * 128
    W16 = B.weights16(params)
    bias = [np.asarray(b, np.float32) for _, b in params]
    K_in = [mlp.IN_PAD] + [mlp.HIDDEN] * 4
    H = [_buffer(lib, s, 0, l, (R, K_in[l]), np.uint16) for l in range(5)]
    Z = [None] + [_buffer(lib, s, 1, l, (R, mlp.HIDDEN), np.float32) for l in range(1, 5)]
    Y = _buffer(lib, s, 2, 0, (R, mlp.OUT_PAD), np.float32)
    dY = _buffer(lib, s, 3, 0, (R, mlp.OUT_PAD), np.uint16)
    dZ32 = [None] + [_buffer(lib, s, 4, l, (R, mlp.HIDDEN), np.float32) for l in range(1, 5)]
    dZ16 = [None] + [_buffer(lib, s, 5, l, (R, mlp.HIDDEN), np.uint16) for l in range(1, 5)]
    x = np.zeros((R, mlp.IN_PAD), np.float32)
    x[:n, :mlp.IN_DIM] = (theta - xm) / xs
    assert np.array_equal(H[0], B.bf16_round64(x))
    # forward: Z_{l+1} = H_l W_l^T + b_l (the saved pre-activation includes the bias)
    for l in range(5):
        pre = Z[l + 1] if l < 4 else Y
        N = pre.shape[1]
        ref = H[l] @ W16[l][:N].T + bias[l][:N]
        S = np.abs(H[l]) @ np.abs(W16[l][:N]).T
        tol = B.gamma(K_in[l]) * S + B.U32 * np.abs(ref) * 2 + 1e-38
        assert np.all(np.abs(pre - ref) <= tol), (l, float((np.abs(pre - ref) / tol).max()))
        if l < 4:
            u = mlp.gelu(pre)
            B.check_rounded(H[l + 1], u, B.fn_err(pre, u) + B.U32 * np.abs(u), f"h{l + 1}")
    # loss gradient dY = bf16(2 w (y - t) / n), from the GPU's own y (FP32 arithmetic as the kernel)
    t32 = np.zeros((R, mlp.OUT_PAD), np.float32)
    t32[:n, :mlp.OUT_DIM] = t
    w32 = np.zeros(mlp.OUT_PAD, np.float32)
    w32[:mlp.OUT_DIM] = w
    d32 = (np.float32(2.0) * w32[None, :] * (Y.astype(np.float32) - t32) / np.float32(n))
    d32[n:] = 0.0
    B.check_rounded(dY, d32.astype(np.float64), 4 * B.U32 * np.abs(d32.astype(np.float64)), "dY")
    loss_ref = float(np.sum((w32[None, :] * (Y.astype(np.float32) - t32) ** 2)[:n].astype(np.float64)) / n)
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    # back-propagation: dZ_l = (dZ_{l+1} W_{l}) * gelu'(Z_l), dZ_5 := dY
    up = {5: dY}
    for l in range(4, 0, -1):
        g_in = up[l + 1]
        Wl = W16[l]                       # [N_l][K_l]: dX_l = dZ_{l+1} W_l
        K = Wl.shape[0]
        acc = g_in[:, :K] @ Wl
        S = np.abs(g_in[:, :K]) @ np.abs(Wl)
        gp = mlp.gelu_grad(Z[l])
        ref = acc * gp
        tol = (np.abs(gp) * B.gamma(K) * S + np.abs(acc) * B.fn_err(Z[l], gp) +
               B.U32 * np.abs(ref) + 1e-38)
        assert np.all(np.abs(dZ32[l] - ref) <= tol), (l, float((np.abs(dZ32[l] - ref) / tol).max()))
        assert np.array_equal(dZ16[l], B.bf16_round64(dZ32[l])), l
        up[l] = dZ16[l]
    # weight and bias gradients
    gpu = surrogate.unflatten(s.last_grads(), mlp.LAYERS)
    chunks = R // (256 if R % 256 == 0 else 128)
    for l in range(5):
        dz = up[l + 1][:, :params[l][0].shape[0]]            # [R][N_l]
        ref = dz.T @ H[l]
        S = np.abs(dz).T @ np.abs(H[l])
        tol = B.gamma(R + chunks) * S + 1e-38
        err = np.abs(gpu[l][0].astype(np.float64) - ref)
        assert np.all(err <= tol), (l, float((err / tol).max()))
        col = (dY[:, :mlp.OUT_PAD] if l == 4 else dZ32[l + 1])
        ref_b = col.sum(axis=0)
        tol_b = B.gamma(R) * np.abs(col).sum(axis=0) + 1e-38
        err_b = np.abs(gpu[l][1].astype(np.float64) - ref_b)
        assert np.all(err_b <= tol_b), (l, float((err_b / tol_b).max()))
    # padding stays zero after the Adam step
    wts = surrogate.unflatten(s.get_weights(), mlp.LAYERS)
    assert np.all(wts[0][0][:, mlp.IN_DIM:] == 0) and np.all(wts[4][0][mlp.OUT_DIM:] == 0)
    assert np.all(wts[4][1][mlp.OUT_DIM:] == 0)


@pytest.mark.parametrize("n", [130, 512])
def test_surrogate_train_step_gradients_match_oracle_within_derived_bound(lib, n):
    """End to end: the weight and bias gradients of one training step against
    the oracle's own (mlp.forward, mlp.loss_and_dy, mlp.backward), element by
    element.  dW_l = dz_l^T x_l: the bound carries the flips of both BF16
    operands (x_l from the forward pass, dz_l from the back-propagation) plus
    each side's accumulation bound; db_l sums the FP32 dz_l.  The flips at
    every rounding point must stay below 1%."""
    from paper_2510_11077_gb300 import surrogate
    s, params, theta, xm, xs, ym, ys, t, w, loss = _train_setup(lib, 17 + n, n)
    R = ((n + 127) // 128) * 128
    gpu = surrogate.unflatten(s.last_grads(), mlp.LAYERS)
    K_in = [mlp.IN_PAD] + [mlp.HIDDEN] * 4
    H = [_buffer(lib, s, 0, l, (R, K_in[l]), np.uint16)[:n] for l in range(5)]
    dY = _buffer(lib, s, 3, 0, (R, mlp.OUT_PAD), np.uint16)[:n]
    dZ32 = [None] + [_buffer(lib, s, 4, l, (R, mlp.HIDDEN), np.float32)[:n] for l in range(1, 5)]
    dZ16 = [None] + [_buffer(lib, s, 5, l, (R, mlp.HIDDEN), np.uint16)[:n] for l in range(1, 5)]
    x, y, cache, _, _ = _oracle_io(params, theta, xm, xs, ym, ys)
    loss_o, dy = mlp.loss_and_dy(y, t, w)
    ref, dz_o, dz32_o = mlp.backward(params, cache, dy, return_dz=True)
    xs_o = cache[0]
    assert abs(loss - loss_o) <= 1e-3 * loss_o
    dx = [np.zeros((n, mlp.IN_PAD))] + [B.flips(H[l], xs_o[l], f"h{l}") for l in range(1, 5)]
    # GPU dZ_{l+1} (the gradient of the pre-activation feeding H_{l+1}) is the
    # oracle's dz of weight layer l; dY that of layer 4
    dz_g = [dZ16[l + 1] for l in range(4)] + [dY]
    dz32_g = [dZ32[l + 1] for l in range(4)] + [dY]
    dd = [B.flips(dz_g[l], dz_o[l], f"dz{l}") for l in range(5)]
    chunks = R // (256 if R % 256 == 0 else 128)
    for l in range(5):
        N = params[l][0].shape[0]
        a_g = dz_g[l][:, :N]
        a_o = dz_o[l][:, :N].astype(np.float64)
        d_dz = dd[l][:, :N]
        Xg, Xo = H[l], xs_o[l].astype(np.float64)
        S_g = np.abs(a_g).T @ np.abs(Xg)
        S_o = np.abs(a_o).T @ np.abs(Xo)
        T = d_dz.T @ np.abs(Xo) + np.abs(a_g).T @ dx[l] + B.gamma(R + chunks) * S_g + B.gamma(n) * S_o
        err = np.abs(gpu[l][0].astype(np.float64) - ref[l][0].astype(np.float64))
        assert np.all(err <= T + 1e-30), (l, float((err / (T + 1e-30)).max()), int(np.sum(err > T)))
        p_g = dz32_g[l][:, :N]
        p_o = dz32_o[l][:, :N].astype(np.float64)
        Tb = np.abs(p_g - p_o).sum(axis=0) + B.gamma(R) * np.abs(p_g).sum(axis=0) + \
            B.gamma(n) * np.abs(p_o).sum(axis=0)
        err_b = np.abs(gpu[l][1].astype(np.float64) - ref[l][1].astype(np.float64))
        assert np.all(err_b <= Tb + 1e-30), (l, float((err_b / (Tb + 1e-30)).max()))


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


def test_training_is_deterministic_on_any_stream(lib):
    """A training step forks its weight-gradient work onto a stream the handle
    owns and joins it back; the same seeded steps on the default stream and on
    a side stream (with other work queued on the default stream meanwhile)
    give bit-identical weights, and a second run on the default stream too."""
    from paper_2510_11077_gb300 import surrogate
    rng = np.random.default_rng(11)
    n = 2500
    theta = rng.standard_normal((n, mlp.IN_DIM)).astype(np.float32)
    ll = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal((n, mlp.IN_DIM)).astype(np.float32)
    th, l_, g_ = (torch.from_numpy(a).cuda() for a in (theta, ll, g))

    def run(stream):
        s = surrogate.Surrogate(device=0, max_rows=4096, seed=5)
        s.set_normalizers(np.zeros(mlp.IN_DIM), np.ones(mlp.IN_DIM), 0.0, 1.0)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            busy = torch.empty(1 << 24, device="cuda")
            for i in range(6):
                busy.normal_()          # unrelated work on the same stream between steps
                s.train_step(th, l_, g_, lr=1e-3)
        torch.cuda.synchronize()
        s.check()
        w = s.get_weights()
        s.close()
        return w

    w0 = run(torch.cuda.default_stream())
    w1 = run(torch.cuda.Stream())
    w2 = run(torch.cuda.default_stream())
    assert np.array_equal(w0, w1)
    assert np.array_equal(w0, w2)


@pytest.mark.parametrize("n", [1, 127, 130, 1000, 2500])
@pytest.mark.parametrize("mode", ["value", "gradient head", "value backprop"])
@pytest.mark.parametrize("baseline", [False, True])
@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_fused_eval_matches_layer_by_layer(lib, n, mode, baseline, cluster):
    """The fused kernel (all layers, and the value output's back-propagation,
    in one launch per 1024 rows, with clusters of 1, 2 or 4 CTAs per slab)
    against the one-GEMM-per-layer path on the same weights and inputs.  Both
    take the same BF16 operands and the same FP32 accumulation order in the
    tensor cores, so they agree to the rounding of a few FP32 operations in
    the epilogues and the baseline's sum: within 1e-4 of the largest
    magnitude.  (Each is held to the oracle itself by the tests above.)"""
    s, params, theta, xm, xs, ym, ys = _setup(20 + n, n)
    if baseline:
        rng = np.random.default_rng(n)
        A = rng.standard_normal((mlp.IN_DIM, mlp.IN_DIM)).astype(np.float32) / mlp.IN_DIM
        s.set_baseline(A @ A.T + 0.1 * np.eye(mlp.IN_DIM, dtype=np.float32))
    if mode == "value backprop":
        s.set_grad_mode(1)
    s.set_cluster(cluster)
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
