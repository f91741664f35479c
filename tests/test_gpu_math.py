"""Accuracy of the device arithmetic that replaces FP64 transcendentals on the
filter's hot path, against CUDA's own functions and high-precision references."""
from __future__ import annotations

import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
try:
    import mpmath
except ImportError:   # not installed on every box; the numpy reference still runs
    mpmath = None


@pytest.fixture(scope="module")
def lib():
    from paper_2510_11077_gb300 import argus
    lib = argus.load()
    dp = ctypes.c_void_p
    lib.argus_selftest_phase.argtypes = [dp, ctypes.c_int64, dp, dp, dp, dp]
    lib.argus_selftest_rcp.argtypes = [dp, ctypes.c_int64, dp]
    lib.argus_selftest_rcp3.argtypes = [dp, ctypes.c_int64, dp]
    lib.argus_selftest_logsum.argtypes = [dp, ctypes.c_int64, dp, dp]
    return lib


def _p(a):
    return a.ctypes.data


def test_phase_sincos_accuracy(lib):
    rng = np.random.default_rng(0)
    # phases a pulsar filter meets: f t + Phi0/2pi up to ~35 cycles, both signs,
    # plus table nodes, half-nodes, tiny and integer phases
    x = np.concatenate([rng.uniform(-40, 40, 20000), rng.uniform(0, 1, 5000),
                        np.arange(0, 3, 1 / 512), [0.0, -0.0, 1e-300, 5e-17, 1.0, -3.0, 33.25],
                        rng.uniform(0, 1e-6, 100)])
    n = len(x)
    s, c, rs, rc = (np.empty(n) for _ in range(4))
    assert lib.argus_selftest_phase(_p(x), n, _p(s), _p(c), _p(rs), _p(rc)) == 0
    # against CUDA's sincospi
    assert np.max(np.abs(s - rs)) < 6e-16 and np.max(np.abs(c - rc)) < 6e-16
    # against numpy on the exact fraction (argument error <= 1 ulp of pi)
    fr = x - np.rint(x)
    assert np.max(np.abs(s - np.sin(2 * np.pi * fr))) < 1.5e-15
    assert np.max(np.abs(c - np.cos(2 * np.pi * fr))) < 1.5e-15
    if mpmath is not None:   # 40-digit reference on a subsample
        mpmath.mp.dps = 40
        idx = rng.choice(n, 1500, replace=False)
        es = max(abs(float(mpmath.sinpi(2 * mpmath.mpf(x[i]))) - s[i]) for i in idx)
        ec = max(abs(float(mpmath.cospi(2 * mpmath.mpf(x[i]))) - c[i]) for i in idx)
        assert es < 5e-16 and ec < 5e-16, (es, ec)
    assert np.all(np.abs(s) <= 1.0 + 1e-15) and np.all(np.abs(c) <= 1.0 + 1e-15)


def _rcp_inputs():
    rng = np.random.default_rng(1)
    return np.concatenate([10.0 ** rng.uniform(-300, 300, 20000), 1e-14 * rng.uniform(0.5, 4, 20000),
                           1.0 + rng.uniform(0.0, 1.0, 20000),
                           [1.0, 2.0, 3.0, 0.1, 2.2250738585072014e-308 * 4, np.nextafter(2.0, 1.0)]])


def test_refined_reciprocal_is_correctly_rounded(lib):
    """The filter kernels' 1/S: a double-float seed (about 2^-44) and one FP64
    Newton step leave (1/S)(1 - e^2), e^2 < 2^-86, so only the last rounding
    remains: within half an ulp of 1/S, up to that 2^-86."""
    S = _rcp_inputs()
    out = np.empty_like(S)
    assert lib.argus_selftest_rcp(_p(S), len(S), _p(out)) == 0
    ref = 1.0 / S
    ulps = np.abs(out - ref) / np.spacing(np.abs(ref))
    assert ulps.max() <= 1.0
    # numpy's division is correctly rounded: the two agree but for ties within 2^-86
    assert np.mean(out == ref) >= 0.9999, np.mean(out == ref)


def test_refined_reciprocal_special_inputs(lib):
    """Negative normal S is the mirror image; zero, subnormal, infinite and NaN
    S take the division (1/S exactly); a reciprocal below the normal range
    (S above 2^1022) flushes to zero, as the approximate instruction does."""
    S = np.array([-3.0, -1e-14, -2.5e300, 0.0, -0.0, 5e-324, 1e-310, np.inf, -np.inf, np.nan,
                  2.0 ** 1023, 1.5 * 2.0 ** 1022, 2.0 ** 1022])
    out = np.empty_like(S)
    assert lib.argus_selftest_rcp(_p(S), len(S), _p(out)) == 0
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / S
    neg = S[:3]
    ulps = np.abs(out[:3] - ref[:3]) / np.spacing(np.abs(ref[:3]))
    assert ulps.max() <= 1.0 and np.all(np.sign(out[:3]) == np.sign(neg))
    assert np.array_equal(out[3:10], ref[3:10], equal_nan=True)
    assert out[10] == 0.0 and out[11] == 0.0
    assert out[12] == 2.0 ** -1022


def test_short_latency_reciprocal_is_within_one_ulp(lib):
    """The scan's and the joint filter's 1/S: the approximate reciprocal and
    one third-order step, (1/S)(1 - e^3) with e^3 < 2^-59."""
    S = _rcp_inputs()
    out = np.empty_like(S)
    assert lib.argus_selftest_rcp3(_p(S), len(S), _p(out)) == 0
    ref = 1.0 / S
    ulps = np.abs(out - ref) / np.spacing(np.abs(ref))
    assert ulps.max() <= 1.0


def test_log_product_matches_sum_of_logs(lib):
    rng = np.random.default_rng(2)
    S = 1e-14 * rng.uniform(0.3, 3.0, 20000)
    out = np.empty(1); bad = np.zeros(1, dtype=np.int32)
    assert lib.argus_selftest_logsum(_p(S), len(S), _p(out), _p(bad)) == 0
    ref = math.fsum(np.log(S))
    assert bad[0] == 0
    assert abs(out[0] - ref) <= 1e-14 * abs(ref)
    for badval in (0.0, -1e-14, np.inf, np.nan, 1e-320):
        T = S[:50].copy(); T[17] = badval
        assert lib.argus_selftest_logsum(_p(T), len(T), _p(out), _p(bad)) == 0
        assert bad[0] == 1, badval


def test_log_product_has_no_overflow_at_the_ends_of_the_double_range(lib):
    """Huge and tiny (but normal) innovation variances: S_k's exponent goes to
    the integer before its mantissa is multiplied in, so the running product
    stays finite and the sum is right, with no false 'bad' flag."""
    rng = np.random.default_rng(3)
    S = np.concatenate([np.array([1.7976931348623157e308, 1.5e308, 2.2250738585072014e-308,
                                  3e-308, 1e308, 1e-307]),
                        10.0 ** rng.uniform(-307, 308, 4000)])
    out = np.empty(1); bad = np.zeros(1, dtype=np.int32)
    assert lib.argus_selftest_logsum(_p(S), len(S), _p(out), _p(bad)) == 0
    assert bad[0] == 0
    ref = math.fsum(np.log(S))
    assert abs(out[0] - ref) <= 1e-13 * np.sum(np.abs(np.log(S))), (out[0], ref)
