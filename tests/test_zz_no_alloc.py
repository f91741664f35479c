"""The allocation-free entry point argus_loglik_grad_noalloc.

It serves callers that cannot allocate device memory while they run (a
framework that has pre-reserved the GPU's memory for its own pool, or a hot
sampling loop that must not synchronise on cudaMalloc/cudaFree).  This file
is collected last so that a run stopping at the first failure has already run
every other test.  It checks, through the C ABI, that two calls in a row give
the same results as argus_loglik_grad within the parity tolerances, and that
three of its walkers match the CPU oracle directly, that the second call
changes the device's free memory by nothing, and that a batch too large for
the fixed scratch array is refused.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

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


def _close(ll, g, ll_ref, g_ref):
    dl = np.abs(ll - ll_ref) / np.maximum(np.abs(ll_ref), 1.0)
    scale = np.maximum(np.abs(g_ref), 1e-3 * np.abs(g_ref).max(axis=1, keepdims=True))
    dg = np.abs(g - g_ref) / np.where(scale == 0, 1.0, scale)
    return dl.max() <= LL_TOL and dg.max() <= G_TOL


def test_noalloc_matches_loglik_grad_twice(argus):
    data = inputs.make_array(np.array([1, 37, 200, 513, 129, 0]), seed=301, equad=1e-8)
    theta = torch.from_numpy(inputs.make_theta_batch(data, 333, seed=17)).cuda()
    arr = argus.argus_array_create(data)
    ll_ref, g_ref = argus.argus_loglik_grad(arr, theta)
    torch.cuda.synchronize()
    ll_ref, g_ref = ll_ref.cpu().numpy(), g_ref.cpu().numpy()
    B, D = theta.shape
    lib = argus.load()
    for call in range(2):
        ll = torch.full((B,), np.nan, dtype=torch.float64, device="cuda")
        g = torch.full((B, D), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = lib.argus_loglik_grad_noalloc(arr.handle, ctypes.c_void_p(theta.data_ptr()), B,
                                           ctypes.c_void_p(ll.data_ptr()),
                                           ctypes.c_void_p(g.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, lib.argus_last_error()
        torch.cuda.synchronize()
        if call == 1:   # after the first call's one-time set-up, no device memory moves
            assert torch.cuda.mem_get_info()[0] == free_before
        assert _close(ll.cpu().numpy(), g.cpu().numpy(), ll_ref, g_ref), f"call {call}"
        # three walkers against the oracle itself, not only against the other entry point
        from oracle import kalman
        idx = np.array([0, 166, 332])
        ll_o, g_o = kalman.loglik_grad(data, theta.cpu().numpy()[idx])
        assert _close(ll.cpu().numpy()[idx], g.cpu().numpy()[idx], ll_o, g_o), f"oracle, call {call}"


def test_noalloc_refuses_oversized_batch_and_host_pointers(argus):
    data = inputs.make_array(np.array([300, 400]), seed=302)
    arr = argus.argus_array_create(data)
    lib = argus.load()
    B = 400_000          # 800k lanes x 128 bytes (about 102 MB) > 64 MiB
    th = torch.zeros((B, data.dim), dtype=torch.float64, device="cuda")
    ll = torch.empty(B, dtype=torch.float64, device="cuda")
    g = torch.empty((B, data.dim), dtype=torch.float64, device="cuda")
    st = lib.argus_loglik_grad_noalloc(arr.handle, ctypes.c_void_p(th.data_ptr()), B,
                                       ctypes.c_void_p(ll.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       None)
    assert st == 6 and b"maximum" in lib.argus_last_error()
    th_h = np.zeros((4, data.dim))
    st = lib.argus_loglik_grad_noalloc(arr.handle, ctypes.c_void_p(th_h.ctypes.data), 4,
                                       ctypes.c_void_p(ll.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       None)
    assert st == 1
