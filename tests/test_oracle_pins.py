"""Pins of the CPU oracle against facts other than itself.

Every check here ties the oracle to mathematics that does not pass through
its own code: the dense Gaussian density (a different algorithm), exact
rational arithmetic, the SDE simulated by Monte Carlo, textbook special cases,
finite differences, closed-form invariants of the antenna patterns, and the
statistical calibration of the innovations.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np
import pytest
from scipy import stats

from oracle import dense, exact, kalman
from paper_2510_11077_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def small_array(sizes, seed, equad=0.0, with_signal=True):
    return inputs.make_array(np.array(sizes), seed=seed, with_signal=with_signal, equad=equad)


# --------------------------------------------------------------------------
# Kalman recursion == dense multivariate normal (prediction-error decomposition)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("kind", ["posterior", "prior"])
def test_kalman_equals_dense_mvn(seed, kind):
    d = small_array([300, 37, 128], seed=seed, equad=3e-8 if seed == 2 else 0.0)
    th = inputs.make_theta_batch(d, 4, seed=seed + 10, kind=kind)
    ll_k = kalman.loglik(d, th)
    ll_d = dense.loglik(d, th)
    rel = np.abs(ll_k - ll_d) / np.maximum(np.abs(ll_d), 1.0)
    assert rel.max() <= 1e-10, rel


def test_kalman_equals_dense_mvn_vs_scipy_logpdf():
    """The dense oracle's Cholesky arithmetic against scipy's own MVN density."""
    d = small_array([60], seed=4)
    th = inputs.make_theta_batch(d, 1, seed=3)[0]
    t, r, sig = d.pulsar(0)
    sig2 = 10.0 ** (2 * th[7])
    R = th[8] ** 2 * sig ** 2
    C = dense.ibm_covariance(t, sig2, d.p0[0], R)
    s = dense.cw_signal(th[:7], d.pos[0], t)
    ref = stats.multivariate_normal(mean=s, cov=C, allow_singular=False).logpdf(r)
    assert abs(kalman.loglik(d, th)[0] - ref) <= 1e-9 * abs(ref)


def test_prediction_error_decomposition_exact_rational():
    """prod S_k = det C and sum e_k^2/S_k = r^T C^-1 r, against exact fractions."""
    rng = np.random.default_rng(7)
    for n in (1, 2, 3, 5, 8):
        t = np.sort(rng.integers(0, 10_000, n)).astype(float) * 1000.0
        t -= t[0]
        r = rng.integers(-300, 300, n) * 1e-9
        sigma = np.full(n, 1e-7)
        p0 = np.array([1e-14, 1e-23, 1e-30])
        sig2, efac = 1e-38, 1.25
        lane = np.array([0.0, 0.0, 1e-8, 0.0, sig2, efac])
        ll, e, S = kalman.pulsar_filter(t, r, sigma, 0.0, p0, lane, trace=True)
        R = [Fr(efac) ** 2 * Fr(1e-7) ** 2] * n
        C = exact.covariance([Fr(x) for x in t], Fr(sig2), [Fr(x) for x in p0], R)
        det, quad = exact.det_and_quad(C, [Fr(x) for x in r])
        logdet = math.log(det.numerator) - math.log(det.denominator)
        assert abs(np.sum(np.log(S)) - logdet) <= 1e-12 * abs(logdet)
        assert abs(np.sum(e * e / S) - float(quad)) <= 1e-11 * max(float(quad), 1.0)
        ll_exact = -0.5 * (float(quad) + logdet + n * math.log(2 * math.pi))
        assert abs(ll - ll_exact) <= 1e-12 * abs(ll_exact)


def test_golden_exact_fixture():
    """Stored exact-rational brute-force values (tests/golden/exact_tiny.json)."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "exact_tiny.json")
    cases = json.load(open(path))["cases"]
    assert len(cases) >= 3
    for c in cases:
        t = np.array(c["t"]); r = np.array(c["r"]); sigma = np.array(c["sigma"])
        lane = np.array([0.0, 0.0, 1e-8, 0.0, c["sig2"], c["efac"]])
        ll = kalman.pulsar_filter(t, r, sigma, c["equad"], np.array(c["p0"]), lane)
        assert abs(ll - c["loglik"]) <= 1e-12 * abs(c["loglik"]), (c["name"], ll, c["loglik"])


def test_white_noise_limit_is_independent_gaussians():
    """sigma_p -> 0 and P0 = 0: ll = sum_k log N(r_k - s_k; 0, R_k) (textbook)."""
    d = small_array([400, 90], seed=11, equad=2e-8)
    d.p0[:] = 0.0
    th = inputs.make_theta_batch(d, 2, seed=5)
    th[:, 7::2] = -400.0          # sigma_p^2 = 10^-800 = 0 in FP64
    ref = []
    for row in th:
        tot = 0.0
        for p in range(d.n_pulsars):
            t, r, sig = d.pulsar(p)
            s = dense.cw_signal(row[:7], d.pos[p], t)
            R = row[8 + 2 * p] ** 2 * sig ** 2 + d.equad[p] ** 2
            tot += stats.norm.logpdf(r - s, scale=np.sqrt(R)).sum()
        ref.append(tot)
    ll = kalman.loglik(d, th)
    assert np.allclose(ll, ref, rtol=1e-12, atol=0)


def test_single_toa_closed_form():
    """N = 1: ll = log N(r - s; 0, P0_rr + R)."""
    t = np.array([0.0]); r = np.array([3e-7]); sigma = np.array([1e-7])
    p0 = np.array([2e-14, 0.0, 1e-32])
    lane = np.array([1e-7, -2e-7, 1e-8, 0.3, 1e-40, 1.1])
    s = lane[0] * math.sin(lane[3]) + lane[1] * math.cos(lane[3])
    ref = stats.norm.logpdf(r[0] - s, scale=math.sqrt(p0[0] + 1.21e-14))
    assert abs(kalman.pulsar_filter(t, r, sigma, 0.0, p0, lane) - ref) <= 1e-13 * abs(ref)


# --------------------------------------------------------------------------
# The process-noise covariance against the SDE itself (Monte Carlo)
# --------------------------------------------------------------------------
def test_ibm_covariance_matches_sde_monte_carlo():
    """d rho/dt = y, dy/dt = xi: Euler-Maruyama ensemble vs the closed form used
    by the dense oracle (and hence the filter's Q)."""
    rng = np.random.default_rng(3)
    n_paths, n_steps, T, sig = 40_000, 400, 2.0, 1.3
    h = T / n_steps
    y = np.zeros(n_paths); rho = np.zeros(n_paths)
    snaps = {100: None, 250: None, 400: None}
    hist = {}
    for k in range(1, n_steps + 1):
        dW = rng.standard_normal(n_paths) * math.sqrt(h)
        rho += y * h + 0.5 * sig * dW * h      # trapezoidal integral of y over the step
        y += sig * dW
        if k in snaps:
            hist[k] = rho.copy()
    times = np.array([100, 250, 400]) * h
    C = dense.ibm_covariance(np.concatenate([[0.0], times]), sig ** 2, [0, 0, 0], 0.0)[1:, 1:]
    emp = np.cov(np.stack([hist[k] for k in (100, 250, 400)]))
    assert np.allclose(emp, C, rtol=0.05, atol=0.02 * C.max())


def test_covariance_vs_state_propagation():
    """The closed form against the covariance built by composing the exact
    discrete transition of the same SDE step by step (matrix exponential of the
    drift, integrated diffusion)."""
    rng = np.random.default_rng(1)
    t = np.sort(rng.uniform(0, 3e8, 25)); t -= t[0]
    sig2 = 1e-40
    p0 = np.array([1e-14, 2e-24, 1e-32])
    P0 = np.array([[p0[0], p0[1]], [p0[1], p0[2]]])
    n = len(t)
    covs = []
    Pk = P0.copy()
    for k in range(n):
        if k:
            dt = t[k] - t[k - 1]
            F = np.array([[1.0, dt], [0.0, 1.0]])
            # integrated diffusion: int_0^dt e^{A s} G G^T e^{A^T s} ds by quadrature
            ss = np.linspace(0, dt, 2001)
            Es = np.stack([np.array([[1.0, s], [0.0, 1.0]]) for s in ss])
            integrand = sig2 * Es[:, :, 1:2] @ Es[:, :, 1:2].transpose(0, 2, 1)
            Q = np.trapezoid(integrand, ss, axis=0)
            Pk = F @ Pk @ F.T + Q
        covs.append(Pk.copy())
    C = np.empty((n, n))
    for i in range(n):
        for j in range(i, n):
            Fij = np.array([[1.0, t[j] - t[i]], [0.0, 1.0]])
            C[i, j] = C[j, i] = (Fij @ covs[i])[0, 0]
    Cd = dense.ibm_covariance(t, sig2, p0, 0.0)
    assert np.allclose(C, Cd, rtol=1e-6, atol=0)


# --------------------------------------------------------------------------
# Gradient pins
# --------------------------------------------------------------------------
def _richardson_fd(f, x, j, h):
    def cd(hh):
        xp = x.copy(); xm = x.copy()
        xp[j] += hh; xm[j] -= hh
        return (f(xp) - f(xm)) / (2 * hh)
    return (4 * cd(h / 2) - cd(h)) / 3


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_vs_richardson_finite_differences(seed):
    d = small_array([120, 70], seed=20 + seed, equad=1e-8)
    th = inputs.make_theta_batch(d, 1, seed=seed)[0]
    _, g = kalman.loglik_grad(d, th)
    f = lambda x: kalman.loglik(d, x)[0]
    steps = [1e-7, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4] + [1e-4, 1e-4] * d.n_pulsars
    fd = np.array([_richardson_fd(f, th, j, steps[j]) for j in range(d.dim)])
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert np.max(np.abs(g[0] - fd) / scale) <= 1e-5


def test_gradient_vs_dense_trace_formula():
    d = small_array([150, 60, 90], seed=30, equad=2e-8)
    for kind in ("posterior", "prior"):
        th = inputs.make_theta_batch(d, 1, seed=4, kind=kind)[0]
        _, g = kalman.loglik_grad(d, th)
        gd = dense.grad(d, th)
        scale = np.maximum(np.abs(gd), 1e-3 * np.abs(gd).max())
        assert np.max(np.abs(g[0] - gd) / scale) <= 1e-8


def test_zero_strain_gives_zero_source_gradients():
    d = small_array([200, 50], seed=31)
    th = inputs.make_theta_batch(d, 1, seed=2)[0]
    th[6] = -300.0
    _, g = kalman.loglik_grad(d, th)
    assert np.all(np.abs(g[0, :6]) < 1e-200)
    assert np.all(np.abs(g[0, 7:]) > 0)


# --------------------------------------------------------------------------
# Continuous-wave projection pins
# --------------------------------------------------------------------------
def _antenna(theta_gw, pos):
    A, B, W, _ = kalman.cw_project(theta_gw, pos)
    h0 = 10.0 ** theta_gw[6]
    cosi = theta_gw[3]
    Fp = A * W / (h0 * (1 + cosi ** 2))
    Fx = -B * W / (2 * h0 * cosi)
    return Fp, Fx


def test_antenna_pattern_rotation_and_antipode():
    rng = np.random.default_rng(5)
    for _ in range(20):
        th = inputs.draw_prior(rng, 1, 1)[0][:7]
        th[3] = 0.6
        c = inputs.isotropic_positions(rng, 1)[0]
        fp0, fx0 = _antenna(th, c)
        for dpsi in (0.3, 1.1, 2.0):
            th2 = th.copy(); th2[2] += dpsi
            fp, fx = _antenna(th2, c)
            # (F+, Fx) rotates by 2 psi: norm kept, angle advanced by 2 dpsi
            assert abs(math.hypot(fp, fx) - math.hypot(fp0, fx0)) <= 1e-12 * math.hypot(fp0, fx0)
            rot = np.array([[math.cos(2 * dpsi), math.sin(2 * dpsi)],
                            [-math.sin(2 * dpsi), math.cos(2 * dpsi)]]) @ np.array([fp0, fx0])
            assert np.allclose([fp, fx], rot, rtol=0, atol=1e-12 * math.hypot(fp0, fx0))
        th3 = th.copy(); th3[2] += math.pi / 2
        fp, fx = _antenna(th3, c)
        assert np.allclose([fp, fx], [-fp0, -fx0], atol=1e-12)
        # pulsar opposite to the source: no response
        cd = math.sqrt(1 - th[4] ** 2)
        n = np.array([cd * math.cos(th[5]), cd * math.sin(th[5]), th[4]])
        fp, fx = _antenna(th, -n)
        assert abs(fp) < 1e-14 and abs(fx) < 1e-14


def test_antenna_pattern_textbook_case():
    """Source at the pole, pulsar on the equator, psi = 0: |F+| = 1/2, Fx = 0."""
    th = np.array([-8.0, 0.0, 0.0, 0.5, 1.0, 0.0, -14.0])
    fp, fx = _antenna(th, np.array([1.0, 0.0, 0.0]))
    assert abs(abs(fp) - 0.5) < 1e-15 and abs(fx) < 1e-15
    # pulsar along +y with psi = pi/8: F+ and Fx share the response equally
    th[2] = math.pi / 8
    fp, fx = _antenna(th, np.array([0.0, 1.0, 0.0]))
    assert abs(abs(fp) - abs(fx)) < 1e-15 and abs(math.hypot(fp, fx) - 0.5) < 1e-15


def test_residual_is_time_integral_of_redshift():
    """ds/dt equals the Earth-term redshift z = F+ h+ + Fx hx with
    h+ = h0 (1 + cos^2 i) cos Phi(t), hx = 2 h0 cos i sin Phi(t)."""
    rng = np.random.default_rng(9)
    th = inputs.draw_prior(rng, 1, 1)[0][:7]
    c = inputs.isotropic_positions(rng, 1)[0]
    fp, fx = _antenna(th, c)
    f = 10 ** th[0]; W = 2 * math.pi * f; h0 = 10 ** th[6]; cosi = th[3]
    t = np.linspace(1e7, 2e8, 50)
    dt = 1.0
    ds = (dense.cw_signal(th, c, t + dt) - dense.cw_signal(th, c, t - dt)) / (2 * dt)
    ph = W * t + th[1]
    z = fp * h0 * (1 + cosi ** 2) * np.cos(ph) + fx * 2 * h0 * cosi * np.sin(ph)
    assert np.allclose(ds, z, rtol=1e-6, atol=1e-9 * np.abs(z).max())


def test_c_and_numpy_projection_agree():
    rng = np.random.default_rng(2)
    for _ in range(10):
        th = inputs.draw_prior(rng, 1, 1)[0][:7]
        c = inputs.isotropic_positions(rng, 1)[0]
        a = kalman.cw_project(th, c)
        b = np.array(dense.cw_project(th, c), dtype=float)
        assert np.allclose(a, b, rtol=1e-13, atol=0)


# --------------------------------------------------------------------------
# Statistical calibration of the whole model
# --------------------------------------------------------------------------
def _simulate_exact(t, theta_lane, p0, sigma, pos, theta_gw, rng):
    sig2, efac = theta_lane
    R = efac ** 2 * sigma ** 2
    C = dense.ibm_covariance(t, sig2, p0, R)
    L = np.linalg.cholesky(C)
    return dense.cw_signal(theta_gw, pos, t) + L @ rng.standard_normal(len(t))


def test_innovations_are_standard_normal():
    rng = np.random.default_rng(12)
    n = 600
    t = np.sort(rng.uniform(0, inputs.T_OBS, n)); t -= t[0]
    sigma = np.full(n, 1e-7)
    p0 = np.array(inputs.P0_DEFAULT)
    th_gw = np.array([-8.2, 1.0, 0.4, 0.3, 0.2, 2.0, -13.5])
    pos = inputs.isotropic_positions(rng, 1)[0]
    sig2, efac = 1e-40, 1.1
    A, B, W, phi0 = kalman.cw_project(th_gw, pos)
    z_all = []
    for _ in range(20):
        r = _simulate_exact(t, (sig2, efac), p0, sigma, pos, th_gw, rng)
        _, e, S = kalman.pulsar_filter(t, r, sigma, 0.0, p0, np.array([A, B, W, phi0, sig2, efac]),
                                       trace=True)
        z_all.append(e / np.sqrt(S))
    z = np.concatenate(z_all)
    N = len(z)
    chi2 = float(np.sum(z * z))
    assert abs(chi2 - N) < 5 * math.sqrt(2 * N)
    assert abs(z.mean()) < 5 / math.sqrt(N)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_mean_score_at_truth_is_zero():
    rng = np.random.default_rng(13)
    n = 150
    t = np.sort(rng.uniform(0, inputs.T_OBS, n)); t -= t[0]
    data = inputs.make_array(np.array([n]), seed=1)
    data.t[:] = t
    th = data.theta_true.copy()
    th[7] = -19.5
    sig2 = 10 ** (2 * th[7])
    scores = []
    for _ in range(150):
        data.r[:] = _simulate_exact(t, (sig2, th[8]), data.p0[0], data.sigma, data.pos[0], th[:7], rng)
        _, g = kalman.loglik_grad(data, th)
        scores.append(g[0])
    s = np.array(scores)
    z = s.mean(0) / (s.std(0) / math.sqrt(len(s)))
    assert np.all(np.abs(z) < 4.5), z


# --------------------------------------------------------------------------
# Batch semantics and domain
# --------------------------------------------------------------------------
def test_batch_permutation_and_duplicates():
    d = small_array([90, 40, 60], seed=40)
    th = inputs.make_theta_batch(d, 5, seed=6)
    th[3] = th[1]
    ll = kalman.loglik(d, th)
    assert ll[3] == ll[1]
    assert np.array_equal(ll, np.array([kalman.loglik(d, x)[0] for x in th]))
    perm = [2, 0, 1]
    d2 = inputs.ArrayData(
        off=np.concatenate([[0], np.cumsum(d.n_toa[perm])]),
        t=np.concatenate([d.pulsar(p)[0] for p in perm]),
        r=np.concatenate([d.pulsar(p)[1] for p in perm]),
        sigma=np.concatenate([d.pulsar(p)[2] for p in perm]),
        pos=d.pos[perm], equad=d.equad[perm], p0=d.p0[perm], theta_true=d.theta_true)
    th2 = np.concatenate([th[:, :7]] + [th[:, 7 + 2 * p: 9 + 2 * p] for p in perm], axis=1)
    assert np.allclose(kalman.loglik(d2, th2), ll, rtol=1e-13)


def test_out_of_domain_parameters():
    d = small_array([50, 30], seed=41)
    th = inputs.make_theta_batch(d, 4, seed=7)
    th[0, 8] = 0.0          # EFAC = 0
    th[1, 3] = 1.5          # |cos i| > 1
    th[2, 0] = np.nan
    ll, g = kalman.loglik_grad(d, th)
    assert np.all(np.isneginf(ll[:3])) and np.isfinite(ll[3])
    assert np.all(g[:3] == 0) and np.any(g[3] != 0)
