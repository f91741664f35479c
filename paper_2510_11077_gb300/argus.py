"""Thin Python binding of the C ABI in include/argus.h (ctypes).

Argument marshalling only: every step of the likelihood runs in the CUDA
library.  If libargus.so is missing or no sm_103 device is present the calls
raise; there is no CPU fallback.

Names follow the C ABI: ``argus_array_create``, ``argus_loglik``,
``argus_loglik_grad``, ``argus_lane_loglik``; ``ArgusLoglik`` is the
torch.autograd.Function a gradient-based sampler calls (paper, Functionality:
"Sampler Integration" -- likelihood and gradient for HMC).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ARGUS_MODE_BATCHED = 0
ARGUS_MODE_PLAIN = 1
ARGUS_MODE_SCAN = 2
ARGUS_NOISE_RANDOM_WALK = 0
ARGUS_NOISE_OU = 1
ARGUS_PULSAR_TERM = 2
NOISE_MODELS = {"rw": ARGUS_NOISE_RANDOM_WALK, "ou": ARGUS_NOISE_OU}


def model_flags(data) -> int:
    """argus.h model flags of an ArrayData (red-noise model, pulsar term)."""
    return NOISE_MODELS[getattr(data, "model", "rw")] | \
        (ARGUS_PULSAR_TERM if getattr(data, "pulsar_term", False) else 0)


def model_name(flags: int) -> str:
    """'rw' or 'ou', with '+pt' for the pulsar term."""
    return ("ou" if flags & ARGUS_NOISE_OU else "rw") + ("+pt" if flags & ARGUS_PULSAR_TERM else "")
STATUS = {0: "ARGUS_OK", 1: "ARGUS_ERR_INVALID_ARG", 2: "ARGUS_ERR_CUDA", 3: "ARGUS_ERR_OOM",
          4: "ARGUS_ERR_NONFINITE", 5: "ARGUS_ERR_TIMEOUT", 6: "ARGUS_ERR_UNSUPPORTED"}


class ArgusError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ArgusPulsar(ctypes.Structure):
    _fields_ = [("n_toa", ctypes.c_int64),
                ("t", ctypes.POINTER(ctypes.c_double)),
                ("r", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)),
                ("pos", ctypes.c_double * 3),
                ("equad", ctypes.c_double),
                ("p0", ctypes.c_double * 3)]


class ArgusPlan(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32),
                ("walkers_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32),
                ("ckpt_stride", ctypes.c_int32),
                ("use_graph", ctypes.c_int32),
                ("tape_cache", ctypes.c_int32),
                ("scan_elems", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libargus.so; raises if it is absent (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ArgusError(6, f"{path} is not built; run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.c_void_p
    lib.argus_array_create.argtypes = [ctypes.POINTER(ArgusPulsar), ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(vp)]
    lib.argus_array_create.restype = ctypes.c_int
    lib.argus_array_create_ex.argtypes = [ctypes.POINTER(ArgusPulsar), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.POINTER(vp)]
    lib.argus_array_create_ex.restype = ctypes.c_int
    lib.argus_array_model.argtypes = [vp]
    lib.argus_array_model.restype = ctypes.c_int32
    lib.argus_array_destroy.argtypes = [vp]
    lib.argus_array_destroy.restype = None
    lib.argus_array_dim.argtypes = [vp]
    lib.argus_array_dim.restype = ctypes.c_int32
    lib.argus_array_set_plan.argtypes = [vp, ctypes.POINTER(ArgusPlan)]
    lib.argus_array_set_plan.restype = ctypes.c_int
    lib.argus_array_get_plan.argtypes = [vp, ctypes.POINTER(ArgusPlan)]
    lib.argus_array_get_plan.restype = ctypes.c_int
    lib.argus_loglik.argtypes = [vp, dp, ctypes.c_int64, dp, vp]
    lib.argus_loglik.restype = ctypes.c_int
    lib.argus_loglik_grad.argtypes = [vp, dp, ctypes.c_int64, dp, dp, vp]
    lib.argus_loglik_grad.restype = ctypes.c_int
    lib.argus_lane_loglik.argtypes = [vp, dp, ctypes.c_int64, dp, vp]
    lib.argus_walker_flags.argtypes = [vp, dp, ctypes.c_int64, dp, vp, vp]
    lib.argus_lane_loglik.restype = ctypes.c_int
    lib.argus_loglik_grad_noalloc.argtypes = [vp, dp, ctypes.c_int64, dp, dp, vp]
    lib.argus_loglik_grad_noalloc.restype = ctypes.c_int
    lib.argus_cw_signal.argtypes = [vp, dp, dp]
    lib.argus_cw_signal.restype = ctypes.c_int
    lib.argus_array_set_timing.argtypes = [vp, ctypes.c_int32]
    lib.argus_array_set_timing.restype = ctypes.c_int
    lib.argus_array_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.argus_array_get_timing.restype = ctypes.c_int
    lib.argus_gwb_create.argtypes = [ctypes.POINTER(ArgusPulsar), ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(vp)]
    lib.argus_gwb_create.restype = ctypes.c_int
    lib.argus_gwb_destroy.argtypes = [vp]
    lib.argus_gwb_destroy.restype = None
    lib.argus_gwb_dim.argtypes = [vp]
    lib.argus_gwb_dim.restype = ctypes.c_int32
    lib.argus_gwb_loglik.argtypes = [vp, dp, ctypes.c_int64, dp, vp]
    lib.argus_gwb_loglik.restype = ctypes.c_int
    lib.argus_gwb_loglik_grad.argtypes = [vp, dp, ctypes.c_int64, dp, dp, vp]
    lib.argus_gwb_loglik_grad.restype = ctypes.c_int
    lib.argus_status_string.argtypes = [ctypes.c_int]
    lib.argus_status_string.restype = ctypes.c_char_p
    lib.argus_last_error.argtypes = []
    lib.argus_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int, allow_nonfinite: bool = False) -> None:
    """Raise on a non-OK status.  allow_nonfinite: accept ARGUS_ERR_NONFINITE,
    whose outputs are all written (the failing walkers hold -inf)."""
    if st != 0 and not (allow_nonfinite and st == 4):
        raise ArgusError(st, _lib.argus_last_error().decode())


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_of(*tensors):
    import torch
    for t in tensors:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


def _pulsar_structs(data):
    P = data.n_pulsars
    keep = []
    ps = (ArgusPulsar * P)()
    dp = ctypes.POINTER(ctypes.c_double)
    for p in range(P):
        t, r, s = (np.ascontiguousarray(a, dtype=np.float64) for a in data.pulsar(p))
        keep += [t, r, s]
        ps[p].n_toa = len(t)
        ps[p].t = t.ctypes.data_as(dp)
        ps[p].r = r.ctypes.data_as(dp)
        ps[p].sigma = s.ctypes.data_as(dp)
        ps[p].pos[:] = [float(v) for v in data.pos[p]]
        ps[p].equad = float(data.equad[p])
        ps[p].p0[:] = [float(v) for v in data.p0[p]]
    return ps, keep


class GwbArray:
    """Handle of the joint likelihood with a Hellings-Downs correlated GW
    background (argus_gwb_create, include/argus_gwb.h); theta = [log10 h_a,
    log10 gamma_a, (log10 sigma_p, log10 gamma_p, EFAC_p) per pulsar]."""

    def __init__(self, data, device: int = 0):
        lib = load()
        ps, keep = _pulsar_structs(data)
        h = ctypes.c_void_p()
        _check(lib.argus_gwb_create(ps, data.n_pulsars, device, ctypes.byref(h)))
        self.handle = h
        self.n_pulsars = data.n_pulsars
        self.dim = lib.argus_gwb_dim(h)
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            _lib.argus_gwb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def argus_gwb_loglik(array: GwbArray, theta, loglik=None, stream=None):
    theta = _prep(theta, array.dim)
    B = theta.shape[0]
    if loglik is None:
        loglik = _new_like(theta, (B,))
    s = stream if stream is not None else _stream_of(theta, loglik)
    _check(_lib.argus_gwb_loglik(array.handle, _ptr(theta), B, _ptr(loglik), s))
    return loglik


def argus_gwb_loglik_grad(array: GwbArray, theta, loglik=None, grad=None, stream=None):
    theta = _prep(theta, array.dim)
    B = theta.shape[0]
    if loglik is None:
        loglik = _new_like(theta, (B,))
    if grad is None:
        grad = _new_like(theta, (B, array.dim))
    s = stream if stream is not None else _stream_of(theta, loglik, grad)
    _check(_lib.argus_gwb_loglik_grad(array.handle, _ptr(theta), B, _ptr(loglik), _ptr(grad), s))
    return loglik, grad


class Array:
    """Handle of one pulsar array on one device (argus_array_create_ex; the
    red-noise model is ``data.model``, "rw" or "ou", and ``data.pulsar_term``
    adds the wave's pulsar term)."""

    def __init__(self, data, device: int = 0):
        lib = load()
        model = model_flags(data)
        P = data.n_pulsars
        self._keep = []
        ps = (ArgusPulsar * P)()
        for p in range(P):
            t, r, s = (np.ascontiguousarray(a, dtype=np.float64) for a in data.pulsar(p))
            self._keep += [t, r, s]
            dp = ctypes.POINTER(ctypes.c_double)
            ps[p].n_toa = len(t)
            ps[p].t = t.ctypes.data_as(dp)
            ps[p].r = r.ctypes.data_as(dp)
            ps[p].sigma = s.ctypes.data_as(dp)
            ps[p].pos[:] = [float(v) for v in data.pos[p]]
            ps[p].equad = float(data.equad[p])
            ps[p].p0[:] = [float(v) for v in data.p0[p]]
        h = ctypes.c_void_p()
        _check(lib.argus_array_create_ex(ps, P, device, model, ctypes.byref(h)))
        self._keep = None
        self.handle = h
        self.n_pulsars = P
        self.dim = lib.argus_array_dim(h)
        self.model = lib.argus_array_model(h)
        self.noise_model = self.model & ARGUS_NOISE_OU
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            _lib.argus_array_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, enable: bool) -> None:
        _check(_lib.argus_array_set_timing(self.handle, int(bool(enable))))

    def get_timing(self):
        """(K1, filter, K4) durations of the last timed call, milliseconds."""
        ms = (ctypes.c_float * 3)()
        _check(_lib.argus_array_get_timing(self.handle, ms))
        return tuple(ms)

    def get_plan(self) -> dict:
        p = ArgusPlan()
        _check(_lib.argus_array_get_plan(self.handle, ctypes.byref(p)))
        return dict(mode=p.mode, walkers_per_cta=p.walkers_per_cta, ctas_per_sm=p.ctas_per_sm,
                    ckpt_stride=p.ckpt_stride, use_graph=p.use_graph, tape_cache=p.tape_cache,
                    scan_elems=p.scan_elems)

    def set_plan(self, **kw) -> None:
        cur = self.get_plan()
        cur.update(kw)
        p = ArgusPlan(cur["mode"], cur["walkers_per_cta"], cur["ctas_per_sm"],
                      cur["ckpt_stride"], cur["use_graph"], cur["tape_cache"], cur["scan_elems"], 0)
        _check(_lib.argus_array_set_plan(self.handle, ctypes.byref(p)))


def argus_array_create(data, device: int = 0) -> Array:
    return Array(data, device)


def _new_like(theta, shape):
    if isinstance(theta, np.ndarray):
        return np.empty(shape, dtype=np.float64)
    import torch
    return torch.empty(shape, dtype=torch.float64, device=theta.device)


def _prep(theta, dim):
    if isinstance(theta, np.ndarray):
        theta = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    else:
        if theta.dim() == 1:
            theta = theta[None, :]
        assert theta.dtype.is_floating_point and theta.element_size() == 8, "theta must be float64"
        theta = theta.contiguous()
    if theta.shape[1] != dim:
        raise ArgusError(1, f"theta has {theta.shape[1]} columns, array needs {dim}")
    return theta


def argus_loglik(array: Array, theta, loglik=None, stream=None, strict=False):
    """strict: raise ArgusError on ARGUS_ERR_NONFINITE (host outputs and a
    walker whose filter failed) instead of returning its -inf."""
    theta = _prep(theta, array.dim)
    B = theta.shape[0]
    if loglik is None:
        loglik = _new_like(theta, (B,))
    s = stream if stream is not None else _stream_of(theta, loglik)
    _check(_lib.argus_loglik(array.handle, _ptr(theta), B, _ptr(loglik), s), not strict)
    return loglik


def argus_loglik_grad(array: Array, theta, loglik=None, grad=None, stream=None, strict=False):
    theta = _prep(theta, array.dim)
    B = theta.shape[0]
    if loglik is None:
        loglik = _new_like(theta, (B,))
    if grad is None:
        grad = _new_like(theta, (B, array.dim))
    s = stream if stream is not None else _stream_of(theta, loglik, grad)
    _check(_lib.argus_loglik_grad(array.handle, _ptr(theta), B, _ptr(loglik), _ptr(grad), s),
           not strict)
    return loglik, grad


def argus_walker_flags(array: Array, theta, loglik, flags=None, stream=None):
    """Per-walker status of a finished call (device tensors): 0 finite, 1 theta
    out of the domain, 2 the filter met a bad innovation variance."""
    import torch
    theta = _prep(theta, array.dim)
    if flags is None:
        flags = torch.empty(theta.shape[0], dtype=torch.int32, device=theta.device)
    s = stream if stream is not None else _stream_of(theta, loglik, flags)
    _check(_lib.argus_walker_flags(array.handle, _ptr(theta), theta.shape[0], _ptr(loglik),
                                   _ptr(flags), s))
    return flags


def argus_loglik_grad_noalloc(array: Array, theta, loglik, grad, stream=None):
    """Allocation-free loglik + gradient: all three tensors must already be on
    the device; the library takes its scratch from a fixed 64 MiB device
    array instead of allocating (see include/argus.h)."""
    theta = _prep(theta, array.dim)
    s = stream if stream is not None else _stream_of(theta, loglik, grad)
    _check(_lib.argus_loglik_grad_noalloc(array.handle, _ptr(theta), theta.shape[0],
                                          _ptr(loglik), _ptr(grad), s))
    return loglik, grad


def argus_cw_signal(array: Array, theta_gw, n_total: int) -> np.ndarray:
    """The model's continuous-wave residual at every TOA (host arrays)."""
    th = np.ascontiguousarray(theta_gw[:7], dtype=np.float64)
    out = np.empty(int(n_total), dtype=np.float64)
    _check(_lib.argus_cw_signal(array.handle, th.ctypes.data, out.ctypes.data))
    return out


def argus_lane_loglik(array: Array, theta, lane=None, stream=None):
    theta = _prep(theta, array.dim)
    B = theta.shape[0]
    if lane is None:
        lane = _new_like(theta, (B, array.n_pulsars))
    s = stream if stream is not None else _stream_of(theta, lane)
    _check(_lib.argus_lane_loglik(array.handle, _ptr(theta), B, _ptr(lane), s))
    return lane


def _autograd_function():
    import torch

    class ArgusLoglik(torch.autograd.Function):
        """loglik(theta) with the adjoint-kernel gradient as its backward."""

        @staticmethod
        def forward(ctx, theta, array):
            ll, g = argus_loglik_grad(array, theta.detach())
            ctx.save_for_backward(g)
            return ll

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout[:, None] * g, None

    return ArgusLoglik


_ArgusLoglik = None


def loglik_autograd(theta, array: Array):
    """Differentiable array log-likelihood: ``ArgusLoglik.apply(theta, array)``."""
    global _ArgusLoglik
    if _ArgusLoglik is None:
        _ArgusLoglik = _autograd_function()
    return _ArgusLoglik.apply(theta, array)
