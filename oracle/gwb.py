"""ctypes wrapper of the joint-likelihood oracle with a Hellings-Downs
correlated GW background (``gwb.c``).  TEST INFRASTRUCTURE ONLY.

theta = [log10 h_a, log10 gamma_a, (log10 sigma_p, log10 gamma_p, EFAC_p)_p].
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import kalman as _k

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def _lib(lib_path=None):
    lib = _k._load(lib_path)
    if not getattr(lib, "_gwb_ready", False):
        arr = [ctypes.c_int, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int64]
        lib.oracle_gwb_loglik.argtypes = arr + [_dp]
        lib.oracle_gwb_loglik.restype = ctypes.c_int
        lib.oracle_gwb_loglik_grad.argtypes = arr + [_dp, _dp]
        lib.oracle_gwb_loglik_grad.restype = ctypes.c_int
        lib.oracle_hellings_downs.argtypes = [ctypes.c_int, _dp, _dp]
        lib.oracle_hellings_downs.restype = None
        lib._gwb_ready = True
    return lib


def dim(data) -> int:
    return 2 + 3 * data.n_pulsars


def _args(data):
    off = np.ascontiguousarray(data.off, dtype=np.int64)
    keep = [off] + [_k._d(a) for a in (data.t, data.r, data.sigma, data.pos, data.equad, data.p0)]
    return keep, [ctypes.c_int(data.n_pulsars), off.ctypes.data_as(_ip)] + [_k._ptr(a) for a in keep[1:]]


def hellings_downs(pos, lib_path=None):
    pos = _k._d(pos)
    P = len(pos)
    G = np.empty((P, P))
    _lib(lib_path).oracle_hellings_downs(P, _k._ptr(pos), _k._ptr(G))
    return G


def loglik(data, theta, lib_path=None):
    lib = _lib(lib_path)
    theta = _k._d(np.atleast_2d(theta))
    B = theta.shape[0]
    out = np.empty(B)
    keep, args = _args(data)
    lib.oracle_gwb_loglik(*args, _k._ptr(theta), ctypes.c_int64(B), _k._ptr(out))
    return out


def loglik_grad(data, theta, lib_path=None):
    lib = _lib(lib_path)
    theta = _k._d(np.atleast_2d(theta))
    B = theta.shape[0]
    ll = np.empty(B)
    g = np.empty((B, theta.shape[1]))
    keep, args = _args(data)
    lib.oracle_gwb_loglik_grad(*args, _k._ptr(theta), ctypes.c_int64(B), _k._ptr(ll), _k._ptr(g))
    return ll, g
