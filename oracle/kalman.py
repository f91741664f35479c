"""ctypes wrapper of the C oracle (``kalman.c``).  TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_libs: dict = {}


def _load(path: str | None = None):
    """Load the oracle library (default: build it from oracle/*.c)."""
    path = path or _build.build()
    if path not in _libs:
        lib = ctypes.CDLL(path)
        arr = [ctypes.c_int, _ip, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int64]
        lib.oracle_loglik.argtypes = arr + [_dp, _dp]
        lib.oracle_loglik.restype = ctypes.c_int
        lib.oracle_loglik_grad.argtypes = arr + [_dp, _dp]
        lib.oracle_loglik_grad.restype = ctypes.c_int
        lib.oracle_cw_project.argtypes = [_dp, _dp, _dp]
        lib.oracle_cw_project.restype = ctypes.c_int
        lib.oracle_pulsar_filter.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                             _dp, _dp, _dp, _dp]
        lib.oracle_pulsar_filter.restype = ctypes.c_double
        _libs[path] = lib
    return _libs[path]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _array_args(data):
    off = np.ascontiguousarray(data.off, dtype=np.int64)
    keep = [off, _d(data.t), _d(data.r), _d(data.sigma), _d(data.pos), _d(data.equad), _d(data.p0)]
    model = (1 if getattr(data, "model", "rw") == "ou" else 0) | \
        (2 if getattr(data, "pulsar_term", False) else 0)
    args = ([ctypes.c_int(data.n_pulsars), off.ctypes.data_as(_ip)] + [_ptr(a) for a in keep[1:]]
            + [ctypes.c_int(model)])
    return keep, args


def set_threads(n: int | None, lib_path: str | None = None) -> int:
    """Number of OpenMP threads the oracle uses (None: leave it); returns the
    number now in effect."""
    lib = _load(lib_path)
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    return int(lib.oracle_set_threads(int(n) if n is not None else 0))


def loglik(data, theta, lanes: bool = False, lib_path: str | None = None):
    """Array log-likelihood float64 [B] (and per-pulsar terms [B, P] if lanes)."""
    lib = _load(lib_path)
    theta = _d(np.atleast_2d(theta))
    B = theta.shape[0]
    assert theta.shape[1] == data.dim
    out = np.empty(B)
    lane = np.empty((B, data.n_pulsars)) if lanes else None
    keep, args = _array_args(data)
    lib.oracle_loglik(*args, _ptr(theta), ctypes.c_int64(B), _ptr(out), _ptr(lane))
    return (out, lane) if lanes else out


def loglik_grad(data, theta, lib_path: str | None = None):
    """(log-likelihood [B], gradient [B, D]) by the complex-step method."""
    lib = _load(lib_path)
    theta = _d(np.atleast_2d(theta))
    B = theta.shape[0]
    assert theta.shape[1] == data.dim
    ll = np.empty(B)
    g = np.empty((B, data.dim))
    keep, args = _array_args(data)
    lib.oracle_loglik_grad(*args, _ptr(theta), ctypes.c_int64(B), _ptr(ll), _ptr(g))
    return ll, g


def cw_project(theta_gw, pos, lib_path: str | None = None, with_delay: bool = False):
    """(A, B, Omega, Phi0) of one parameter vector on one pulsar; with
    with_delay also 1 - n.c (clamped), the pulsar term's geometric factor."""
    lib = _load(lib_path)
    th = _d(theta_gw[:7]); c = _d(pos); out = np.empty(5)
    lib.oracle_cw_project(_ptr(th), _ptr(c), _ptr(out))
    return out if with_delay else out[:4]


def pulsar_filter(t, r, sigma, equad, p0, lane, trace: bool = False,
                  lib_path: str | None = None):
    """One pulsar's log-likelihood for lane = (A, B, Omega, Phi0, sigma^2, EFAC
    [, gamma [, Dp]]); gamma > 0 selects the Ornstein-Uhlenbeck red noise and
    Dp != 0 adds the pulsar term with phase lag Dp (rad).

    With trace=True also returns the innovations e_k and variances S_k.
    """
    lib = _load(lib_path)
    lane = np.concatenate([np.asarray(lane, dtype=np.float64), np.zeros(8 - len(lane))])
    t, r, sigma, p0, lane = _d(t), _d(r), _d(sigma), _d(p0), _d(lane)
    n = len(t)
    e = np.empty(n) if trace else None
    S = np.empty(n) if trace else None
    ll = lib.oracle_pulsar_filter(ctypes.c_int64(n), _ptr(t), _ptr(r), _ptr(sigma),
                                  ctypes.c_double(equad), _ptr(p0), _ptr(lane), _ptr(e), _ptr(S))
    return (ll, e, S) if trace else ll
