"""Thin Python binding of the surrogate network's C ABI
(include/argus_surrogate.h): argument marshalling only, the network runs in
libargus.so on the tensor cores."""
from __future__ import annotations

import ctypes

import numpy as np

from . import argus as _argus

N_IN = 47
N_OUT = 48


class SurrogateError(RuntimeError):
    pass


def _lib():
    lib = _argus.load()
    if not getattr(lib, "_surrogate_ready", False):
        vp = ctypes.c_void_p
        lib.argus_surrogate_param_count.restype = ctypes.c_int64
        lib.argus_surrogate_param_count.argtypes = []
        lib.argus_surrogate_create_ex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                                  ctypes.POINTER(vp)]
        lib.argus_surrogate_create.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(vp)]
        lib.argus_surrogate_save.argtypes = [vp, ctypes.c_char_p]
        lib.argus_surrogate_last_loss.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.argus_surrogate_destroy.argtypes = [vp]
        lib.argus_surrogate_destroy.restype = None
        lib.argus_surrogate_set_normalizers.argtypes = [vp, vp, vp, ctypes.c_float, ctypes.c_float,
                                                        ctypes.c_float, ctypes.c_float]
        lib.argus_surrogate_set_weights.argtypes = [vp, vp]
        lib.argus_surrogate_set_baseline.argtypes = [vp, vp]
        lib.argus_surrogate_set_grad_mode.argtypes = [vp, ctypes.c_int32]
        lib.argus_surrogate_set_fused.argtypes = [vp, ctypes.c_int32]
        lib.argus_surrogate_set_cluster.argtypes = [vp, ctypes.c_int32]
        lib.argus_surrogate_eval_f64.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int64, vp, vp, vp]
        lib.argus_surrogate_get_weights.argtypes = [vp, vp]
        lib.argus_surrogate_eval.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
        lib.argus_surrogate_train_step_ex.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float,
                                                      vp, vp]
        lib.argus_surrogate_train_step.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float, vp]
        lib.argus_surrogate_check.argtypes = [vp]
        lib.argus_surrogate_last_error.restype = ctypes.c_char_p
        lib.argus_selftest_surrogate_grads.argtypes = [vp, vp]
        lib._surrogate_ready = True
    return lib


def _check(st):
    if st != 0:
        raise SurrogateError(f"{_argus.STATUS.get(st, st)}: {_lib().argus_surrogate_last_error().decode()}")


def param_count() -> int:
    return int(_lib().argus_surrogate_param_count())


class Surrogate:
    """argus_surrogate_create_ex / eval / train_step (argus_surrogate_create
    through from_array)."""

    def __init__(self, device: int = 0, max_rows: int = 4096, seed: int = 1, _handle=None):
        lib = _lib()
        h = _handle
        if h is None:
            h = ctypes.c_void_p()
            _check(lib.argus_surrogate_create_ex(device, max_rows, seed, ctypes.byref(h)))
        self.handle = h
        self.device = device
        self.max_rows = max_rows

    @classmethod
    def from_array(cls, array, weights_path=None):
        """argus_surrogate_create: the surrogate of `array` (an argus.Array with
        D = 47), from a file argus_surrogate_save wrote, or freshly initialised."""
        h = ctypes.c_void_p()
        path = None if weights_path is None else str(weights_path).encode()
        _check(_lib().argus_surrogate_create(array.handle, path, ctypes.byref(h)))
        return cls(device=array.device, max_rows=4096, _handle=h)

    def save(self, path):
        _check(_lib().argus_surrogate_save(self.handle, str(path).encode()))

    def close(self):
        if getattr(self, "handle", None):
            _lib().argus_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_normalizers(self, x_mean, x_std, y_mean, y_std, value_weight=1.0, grad_weight=1.0):
        xm = np.ascontiguousarray(x_mean, dtype=np.float32)
        xs = np.ascontiguousarray(x_std, dtype=np.float32)
        _check(_lib().argus_surrogate_set_normalizers(self.handle, xm.ctypes.data, xs.ctypes.data,
                                                      float(y_mean), float(y_std),
                                                      float(value_weight), float(grad_weight)))

    def set_baseline(self, H):
        """ll ~ net(x) - x^T H x / 2 (H: [47, 47]); None removes it."""
        if H is None:
            _check(_lib().argus_surrogate_set_baseline(self.handle, None))
            return
        Hf = np.ascontiguousarray(H, dtype=np.float32)
        assert Hf.shape == (N_IN, N_IN)
        _check(_lib().argus_surrogate_set_baseline(self.handle, Hf.ctypes.data))

    def set_grad_mode(self, mode: int):
        """0: gradient outputs of the network; 1: back-propagated value output."""
        _check(_lib().argus_surrogate_set_grad_mode(self.handle, int(mode)))

    def set_fused(self, on: bool):
        """Evaluate with the fused kernel (True, default) or layer by layer."""
        _check(_lib().argus_surrogate_set_fused(self.handle, 1 if on else 0))

    def set_cluster(self, ctas: int):
        """CTAs of the fused kernel per 128-row slab: 1, 2, 4, or 0 (automatic)."""
        _check(_lib().argus_surrogate_set_cluster(self.handle, int(ctas)))

    def set_weights(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == param_count()
        _check(_lib().argus_surrogate_set_weights(self.handle, flat.ctypes.data))

    def get_weights(self):
        out = np.empty(param_count(), dtype=np.float32)
        _check(_lib().argus_surrogate_get_weights(self.handle, out.ctypes.data))
        return out

    def last_grads(self):
        out = np.empty(param_count(), dtype=np.float32)
        _check(_lib().argus_selftest_surrogate_grads(self.handle, out.ctypes.data))
        return out

    def eval(self, theta, loglik=None, grad=None, with_grad=True, stream=None):
        import torch
        assert theta.is_cuda and theta.dtype == torch.float32 and theta.shape[1] == N_IN
        theta = theta.contiguous()
        B = theta.shape[0]
        if loglik is None:
            loglik = torch.empty(B, dtype=torch.float32, device=theta.device)
        if with_grad and grad is None:
            grad = torch.empty((B, N_IN), dtype=torch.float32, device=theta.device)
        s = stream if stream is not None else torch.cuda.current_stream(theta.device).cuda_stream
        _check(_lib().argus_surrogate_eval(self.handle, theta.data_ptr(), B, loglik.data_ptr(),
                                           grad.data_ptr() if with_grad else None, s))
        return (loglik, grad) if with_grad else loglik

    def eval_z(self, z, centre, offset=0.0, loglik=None, grad=None, with_grad=True, stream=None):
        """Surrogate at float(z - centre), FP64 in and out (argus_surrogate_eval_f64):
        loglik = value + offset (-inf if not finite) and its gradient."""
        import torch
        assert z.is_cuda and z.dtype == torch.float64 and z.shape[1] == N_IN
        assert centre.is_cuda and centre.dtype == torch.float64 and centre.numel() == N_IN
        z = z.contiguous()
        centre = centre.contiguous()
        B = z.shape[0]
        if loglik is None:
            loglik = torch.empty(B, dtype=torch.float64, device=z.device)
        if with_grad and grad is None:
            grad = torch.empty((B, N_IN), dtype=torch.float64, device=z.device)
        s = stream if stream is not None else torch.cuda.current_stream(z.device).cuda_stream
        _check(_lib().argus_surrogate_eval_f64(self.handle, z.data_ptr(), centre.data_ptr(), float(offset), B,
                                               loglik.data_ptr(), grad.data_ptr() if with_grad else None, s))
        return (loglik, grad) if with_grad else loglik

    def train_step(self, theta, loglik, grad, lr, loss_out=None, stream=None):
        """argus_surrogate_train_step_ex: targets in separate arrays; returns the
        loss (device tensor) before the step."""
        import torch
        n = theta.shape[0]
        if loss_out is None:
            loss_out = torch.empty(1, dtype=torch.float32, device=theta.device)
        s = stream if stream is not None else torch.cuda.current_stream(theta.device).cuda_stream
        _check(_lib().argus_surrogate_train_step_ex(self.handle, theta.data_ptr(), loglik.data_ptr(),
                                                    grad.data_ptr(), n, float(lr), loss_out.data_ptr(),
                                                    s))
        return loss_out

    def train_step_packed(self, x, y, lr, stream=None):
        """argus_surrogate_train_step: y [n][48] = (loglik, gradient)."""
        import torch
        assert x.is_contiguous() and y.is_contiguous() and y.shape[1] == N_OUT
        s = stream if stream is not None else torch.cuda.current_stream(x.device).cuda_stream
        _check(_lib().argus_surrogate_train_step(self.handle, x.data_ptr(), y.data_ptr(), x.shape[0],
                                                 float(lr), s))

    def last_loss(self) -> float:
        v = ctypes.c_float()
        _check(_lib().argus_surrogate_last_loss(self.handle, ctypes.byref(v)))
        return float(v.value)

    def check(self):
        _check(_lib().argus_surrogate_check(self.handle))


def flatten(params) -> np.ndarray:
    """Oracle-style [[W, b], ...] -> flat layout of argus_surrogate.h."""
    return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in params]).astype(np.float32)


def unflatten(flat, layers):
    out, o = [], 0
    for k, n in layers:
        W = flat[o:o + n * k].reshape(n, k); o += n * k
        b = flat[o:o + n]; o += n
        out.append([W.copy(), b.copy()])
    return out
