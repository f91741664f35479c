"""Pins of the Ornstein-Uhlenbeck red-noise oracle (paper, Functionality: OU
processes for pulsar-intrinsic red noise).

The frequency deviation obeys dy = -gamma y dt + sigma dW and the residual is
its integral.  The pins tie the dense covariance and the filter's transition to
things fixed independently of the closed forms the oracle uses: the SDE itself
(Monte Carlo), the defining integral (quadrature), Van Loan's matrix
exponential of the linear SDE, the gamma -> 0 limit (the random walk, pinned on
its own), finite differences, and the calibration of the innovations.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import integrate, linalg, stats

from oracle import dense, kalman
from paper_2510_11077_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def ou_array(sizes, seed, log10_gamma=None, equad=2e-8):
    d = inputs.make_array(np.array(sizes), seed=seed, equad=equad, model="ou")
    if log10_gamma is not None:
        d.theta_true[8::3] = log10_gamma
    return d


def _van_loan(dt, gam, sig2):
    """Exact transition F and process noise Q of d(rho, y) = A (rho, y) dt + G dW
    over dt, from one matrix exponential (Van Loan 1978)."""
    A = np.array([[0.0, 1.0], [0.0, -gam]])
    GG = np.array([[0.0, 0.0], [0.0, sig2]])
    M = np.zeros((4, 4))
    M[:2, :2] = -A
    M[:2, 2:] = GG
    M[2:, 2:] = A.T
    E = linalg.expm(M * dt)
    F = E[2:, 2:].T
    return F, F @ E[:2, 2:]


# --------------------------------------------------------------------------
# The dense covariance
# --------------------------------------------------------------------------
def test_ou_covariance_matches_sde_monte_carlo():
    """Euler-Maruyama ensemble of the SDE, started from a correlated prior."""
    rng = np.random.default_rng(5)
    n_paths, n_steps, T, sig, gam = 40_000, 500, 2.5, 1.3, 0.8
    p0 = np.array([0.3, 0.1, 0.5])
    h = T / n_steps
    L0 = np.linalg.cholesky(np.array([[p0[0], p0[1]], [p0[1], p0[2]]]))
    z0 = L0 @ rng.standard_normal((2, n_paths))
    rho, y = z0[0].copy(), z0[1].copy()
    keep = (120, 300, 500)
    hist = {}
    for k in range(1, n_steps + 1):
        dW = rng.standard_normal(n_paths) * math.sqrt(h)
        y_new = y - gam * y * h + sig * dW
        rho += 0.5 * h * (y + y_new)
        y = y_new
        if k in keep:
            hist[k] = rho.copy()
    times = np.array([0.0] + [k * h for k in keep])
    C = dense.ou_covariance(times, sig ** 2, gam, p0, 0.0)[1:, 1:]
    emp = np.cov(np.stack([hist[k] for k in keep]))
    assert np.allclose(emp, C, rtol=0.05, atol=0.02 * C.max())


@pytest.mark.parametrize("gam", [1e-9, 1e-8, 1e-7])
def test_ou_covariance_vs_quadrature(gam):
    """Each red-noise entry against sigma^2 int_0^m g(v) g(v + M - m) dv by
    adaptive quadrature, g(v) = (1 - e^{-gamma v}) / gamma."""
    rng = np.random.default_rng(int(-math.log10(gam)))
    t = np.concatenate([[0.0], np.sort(rng.uniform(0, inputs.T_OBS, 6))])
    sig2 = 1e-40
    C = dense.ou_covariance(t, sig2, gam, np.zeros(3), 0.0)
    g = lambda v: -math.expm1(-gam * v) / gam
    for i in range(len(t)):
        for j in range(i, len(t)):
            m, d = t[i], t[j] - t[i]
            val, _ = integrate.quad(lambda v: g(v) * g(v + d), 0.0, m, epsabs=0, epsrel=1e-12, limit=200)
            assert C[i, j] == pytest.approx(sig2 * val, rel=1e-9, abs=1e-300)


def test_ou_covariance_vs_state_propagation():
    """The closed form against the covariance built by composing the exact
    discrete transitions (Van Loan) from a non-trivial prior."""
    rng = np.random.default_rng(8)
    t = np.sort(rng.uniform(0, 3e8, 30)); t -= t[0]
    sig2, gam = 1e-40, 3e-8
    p0 = np.array([1e-14, 2e-24, 1e-32])
    Pk = np.array([[p0[0], p0[1]], [p0[1], p0[2]]])
    covs = [Pk.copy()]
    for k in range(1, len(t)):
        F, Q = _van_loan(t[k] - t[k - 1], gam, sig2)
        Pk = F @ Pk @ F.T + Q
        covs.append(Pk.copy())
    n = len(t)
    C = np.empty((n, n))
    for i in range(n):
        for j in range(i, n):
            F, _ = _van_loan(t[j] - t[i], gam, sig2)
            C[i, j] = C[j, i] = (F @ covs[i])[0, 0]
    Cd = dense.ou_covariance(t, sig2, gam, p0, 0.0)
    assert np.allclose(Cd, C, rtol=1e-8, atol=0)


def test_ou_covariance_small_gamma_tends_to_random_walk():
    rng = np.random.default_rng(9)
    t = np.sort(rng.uniform(0, 1e8, 12)); t -= t[0]
    p0 = np.array([1e-14, 3e-24, 1e-32])
    for gam, tol in ((1e-12, 1e-3), (1e-13, 1e-4)):
        Cou = dense.ou_covariance(t, 1e-40, gam, p0, 0.0)
        Crw = dense.ibm_covariance(t, 1e-40, p0, 0.0)
        assert np.allclose(Cou, Crw, rtol=tol, atol=0)


def test_ou_stationary_frequency_variance():
    """Long after the start, y has variance sigma^2 / (2 gamma): the residual
    increments over a short lag dt have variance ~ dt^2 sigma^2 / (2 gamma)."""
    gam, sig2, dt = 1e-7, 1e-40, 1e3
    t = np.array([0.0, 3e8, 3e8 + dt])
    C = dense.ou_covariance(t, sig2, gam, np.zeros(3), 0.0)
    var_inc = C[2, 2] + C[1, 1] - 2 * C[1, 2]
    assert var_inc / dt ** 2 == pytest.approx(sig2 / (2 * gam), rel=1e-4)


# --------------------------------------------------------------------------
# The filter
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,lg", [(0, -7.0), (1, -7.6), (2, -8.5), (3, -10.0)])
def test_kalman_ou_equals_dense_mvn(seed, lg):
    d = ou_array([90, 40, 130], seed=40 + seed, log10_gamma=lg)
    th = inputs.make_theta_batch(d, 3, seed=seed)
    ll = kalman.loglik(d, th)
    ref = dense.loglik(d, th)
    assert np.allclose(ll, ref, rtol=1e-10, atol=0)


def test_kalman_ou_spans_series_and_closed_form_steps():
    """With gamma = 1e-7 the steps gamma dt fall on both sides of 0.5, where the
    transition switches from Taylor series to closed forms; the filter must
    agree with the dense likelihood on each side and across the switch."""
    rng = np.random.default_rng(3)
    small = np.cumsum(rng.uniform(1e5, 4e6, 40))
    t = np.concatenate([small, small[-1] + np.cumsum(rng.uniform(4e6, 3e7, 30))])
    x = 1e-7 * np.diff(t)
    assert (x < 0.5).sum() > 10 and (x >= 0.5).sum() > 10
    sigma = np.full(len(t), 1e-7)
    r = 1e-6 * rng.standard_normal(len(t))
    p0 = np.array(inputs.P0_DEFAULT)
    for gam in (1e-7, 1.3e-7, 0.8e-7):
        lane = np.array([0.0, 0.0, 1e-8, 0.0, 1e-39, 1.0, gam])
        ll = kalman.pulsar_filter(t, r, sigma, 0.0, p0, lane)
        C = dense.ou_covariance(t - t[0], 1e-39, gam, p0, sigma ** 2)
        ref = stats.multivariate_normal(mean=np.zeros(len(t)), cov=C).logpdf(r)
        assert ll == pytest.approx(ref, rel=1e-10)


def test_kalman_ou_tiny_gamma_equals_random_walk():
    d = ou_array([70, 50], seed=11, log10_gamma=-20.0)
    th = inputs.make_theta_batch(d, 2, seed=1)
    th[:, 8::3] = -20.0
    rw = inputs.ArrayData(off=d.off, t=d.t, r=d.r, sigma=d.sigma, pos=d.pos, equad=d.equad,
                          p0=d.p0, theta_true=d.theta_true, model="rw")
    th_rw = np.concatenate([th[:, :7]] + [th[:, [7 + 3 * p, 9 + 3 * p]] for p in range(2)], axis=1)
    assert np.allclose(kalman.loglik(d, th), kalman.loglik(rw, th_rw), rtol=1e-12, atol=0)


def test_kalman_ou_innovations_are_standard_normal():
    rng = np.random.default_rng(14)
    n = 500
    t = np.sort(rng.uniform(0, inputs.T_OBS, n)); t -= t[0]
    sigma = np.full(n, 1e-7)
    p0 = np.array(inputs.P0_DEFAULT)
    sig2, efac, gam = 1e-39, 1.05, 2e-8
    C = dense.ou_covariance(t, sig2, gam, p0, (efac * sigma) ** 2)
    L = np.linalg.cholesky(C)
    lane = np.array([0.0, 0.0, 1e-8, 0.0, sig2, efac, gam])
    z_all = []
    for _ in range(20):
        r = L @ rng.standard_normal(n)
        _, e, S = kalman.pulsar_filter(t, r, sigma, 0.0, p0, lane, trace=True)
        z_all.append(e / np.sqrt(S))
    z = np.concatenate(z_all)
    N = len(z)
    assert abs(float(np.sum(z * z)) - N) < 5 * math.sqrt(2 * N)
    assert stats.kstest(z, "norm").pvalue > 1e-4


# --------------------------------------------------------------------------
# Gradients, including d / d log10 gamma
# --------------------------------------------------------------------------
def _richardson_fd(f, x, j, h):
    def cd(hh):
        xp = x.copy(); xm = x.copy()
        xp[j] += hh; xm[j] -= hh
        return (f(xp) - f(xm)) / (2 * hh)
    return (4 * cd(h / 2) - cd(h)) / 3


@pytest.mark.parametrize("lg", [-7.2, -9.0])
def test_ou_gradient_vs_richardson_finite_differences(lg):
    d = ou_array([110, 60], seed=21, log10_gamma=lg, equad=1e-8)
    th = inputs.make_theta_batch(d, 1, seed=2)[0]
    _, g = kalman.loglik_grad(d, th)
    f = lambda x: kalman.loglik(d, x)[0]
    steps = [1e-7] + [1e-4] * (d.dim - 1)
    fd = np.array([_richardson_fd(f, th, j, steps[j]) for j in range(d.dim)])
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert np.max(np.abs(g[0] - fd) / scale) <= 1e-5


def test_ou_gradient_vs_dense_trace_formula():
    d = ou_array([80, 60, 45], seed=31, log10_gamma=-7.5)
    for kind in ("posterior", "prior"):
        th = inputs.make_theta_batch(d, 2, seed=4, kind=kind)
        _, g = kalman.loglik_grad(d, th)
        for b in range(2):
            gd = dense.grad(d, th[b])
            scale = np.maximum(np.abs(gd), 1e-6 * np.abs(gd).max())
            assert np.max(np.abs(g[b] - gd) / scale) <= 1e-7, kind


def test_ou_out_of_domain_parameters():
    d = ou_array([40, 30], seed=42)
    th = inputs.make_theta_batch(d, 3, seed=7)
    th[0, 9] = 0.0          # EFAC = 0 (third noise slot of pulsar 0)
    th[1, 12] = -0.2        # EFAC < 0 of pulsar 1
    ll, g = kalman.loglik_grad(d, th)
    assert np.all(np.isneginf(ll[:2])) and np.isfinite(ll[2])
    assert np.all(g[:2] == 0) and np.all(np.isfinite(g[2]))
    # gamma itself has no lower wall: any real log10 gamma is in the domain
    th[2, 8] = -25.0
    assert np.isfinite(kalman.loglik(d, th[2:])[0])
