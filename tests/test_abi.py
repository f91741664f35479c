"""The C-ABI library builds, loads and exports every declared entry point; its
host-side validation runs without a GPU (no compute calls here)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2510_11077_gb300 import argus, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return argus.load()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(argus_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("argus_array_create", "argus_loglik", "argus_loglik_grad", "argus_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.argus_status_string(0) == b"ARGUS_OK"
    assert lib.argus_status_string(1) == b"ARGUS_ERR_INVALID_ARG"
    assert lib.argus_status_string(99) == b"ARGUS_ERR_UNKNOWN"
    assert lib.argus_array_dim(None) == -1


def _pulsars(data):
    keep = []
    ps = (argus.ArgusPulsar * data.n_pulsars)()
    dp = ctypes.POINTER(ctypes.c_double)
    for p in range(data.n_pulsars):
        t, r, s = (np.ascontiguousarray(a) for a in data.pulsar(p))
        keep += [t, r, s]
        ps[p].n_toa = len(t)
        ps[p].t, ps[p].r, ps[p].sigma = (a.ctypes.data_as(dp) for a in (t, r, s))
        ps[p].pos[:] = list(data.pos[p])
        ps[p].equad = data.equad[p]
        ps[p].p0[:] = list(data.p0[p])
    return ps, keep


@pytest.mark.parametrize("bad", ["unsorted", "sigma0", "nan_r", "pos", "equad", "p0", "count"])
def test_create_rejects_bad_input_before_any_device_call(lib, bad):
    data = inputs.make_array(np.array([20, 30]), seed=1)
    if bad == "unsorted":
        data.t[5], data.t[6] = data.t[6], data.t[5] + 1.0
    elif bad == "sigma0":
        data.sigma[3] = 0.0
    elif bad == "nan_r":
        data.r[10] = np.nan
    elif bad == "pos":
        data.pos[1] *= 1.1
    elif bad == "equad":
        data.equad[0] = -1e-8
    elif bad == "p0":
        data.p0[0] = [1e-14, 1e-15, 1e-32]
    ps, keep = _pulsars(data)
    h = ctypes.c_void_p()
    n = 0 if bad == "count" else data.n_pulsars
    st = lib.argus_array_create(ps, n, 0, ctypes.byref(h))
    assert st == 1, (st, lib.argus_last_error())
    assert h.value is None
    assert lib.argus_last_error() != b""


def test_create_ex_rejects_unknown_model_flags(lib):
    data = inputs.make_array(np.array([20, 30]), seed=1)
    ps, keep = _pulsars(data)
    h = ctypes.c_void_p()
    for bad in (4, 7, -1):
        st = lib.argus_array_create_ex(ps, data.n_pulsars, 0, bad, ctypes.byref(h))
        assert st == 1 and h.value is None
        assert b"model must be" in lib.argus_last_error()
    assert lib.argus_array_model(None) == -1


def test_model_flags_of_array_data():
    d = inputs.make_array(np.array([5, 6]), seed=1, model="ou", pulsar_term=True)
    assert argus.model_flags(d) == argus.ARGUS_NOISE_OU | argus.ARGUS_PULSAR_TERM
    assert argus.model_name(argus.model_flags(d)) == "ou+pt" and d.dim == 7 + 4 * 2


def test_gwb_create_rejects_too_many_pulsars_and_bad_data(lib):
    data = inputs.make_array(np.full(65, 3), seed=2)
    ps, keep = _pulsars(data)
    h = ctypes.c_void_p()
    assert lib.argus_gwb_create(ps, 65, 0, ctypes.byref(h)) == 6 and h.value is None
    assert b"64" in lib.argus_last_error()
    data = inputs.make_array(np.array([10, 10]), seed=3)
    data.sigma[4] = -1.0
    ps, keep = _pulsars(data)
    assert lib.argus_gwb_create(ps, 2, 0, ctypes.byref(h)) == 1 and h.value is None
    assert lib.argus_gwb_dim(None) == -1
    assert lib.argus_gwb_loglik(None, None, 1, None, None) == 1
    assert lib.argus_gwb_loglik_grad(None, None, 1, None, None, None) == 1


def test_calls_on_null_handle_are_rejected(lib):
    assert lib.argus_loglik(None, None, 1, None, None) == 1
    assert lib.argus_array_set_plan(None, None) == 1
    assert lib.argus_array_get_plan(None, None) == 1


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    """The binding refuses to run when libargus.so is absent."""
    monkeypatch.setattr(argus, "_lib", None)
    monkeypatch.setattr(argus._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(argus.ArgusError):
        argus.load()
