"""Pins of the continuous wave's pulsar term in the oracle (the source model
of the paper's cited prior work on pulsar terms).

The wave reaches the pulsar a time tau_p = d_p (1 - n.c) / c before it
reaches the Earth; the timing residual is the integral of the redshift
z(t) = F+ [h+(t) - h+(t - tau_p)] + Fx [hx(t) - hx(t - tau_p)].  The pins tie
the C filter's phase-lag form and the dense oracle's retarded-time form to
each other and to things fixed outside both: the redshift itself (finite
differences of the residual), the light-year value of the parsec, limits
where the pulsar term vanishes or cancels the Earth term, and finite
differences of the likelihood.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import dense, kalman
from paper_2510_11077_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def pt_array(sizes, seed, model="rw", equad=2e-8):
    return inputs.make_array(np.array(sizes), seed=seed, equad=equad, model=model, pulsar_term=True)


def _antenna(th, c):
    sind, al, psi = th[4], th[5], th[2]
    cosd = math.sqrt(1 - sind ** 2)
    n = np.array([cosd * math.cos(al), cosd * math.sin(al), sind])
    u = np.array([math.sin(al), -math.cos(al), 0.0])
    v = np.array([sind * math.cos(al), sind * math.sin(al), -cosd])
    p = math.cos(psi) * u + math.sin(psi) * v
    q = -math.sin(psi) * u + math.cos(psi) * v
    D = 1 - c @ n
    return 0.5 * ((c @ p) ** 2 - (c @ q) ** 2) / D, (c @ p) * (c @ q) / D, D


def test_kiloparsec_light_time():
    """1 pc = 3.261563777 light-years (IAU definitions of the parsec and the
    astronomical unit, Julian year)."""
    ly_per_kpc = dense.KPC_LIGHT_S / (365.25 * 86400.0)
    assert ly_per_kpc == pytest.approx(3261.563777, rel=1e-9)


def test_residual_derivative_is_earth_minus_pulsar_redshift():
    rng = np.random.default_rng(19)
    th = inputs.draw_prior(rng, 1, 1)[0][:7]
    c = inputs.isotropic_positions(rng, 1)[0]
    d_kpc = 1.3
    fp, fx, D = _antenna(th, c)
    tau = d_kpc * dense.KPC_LIGHT_S * D
    f = 10 ** th[0]; W = 2 * math.pi * f; h0 = 10 ** th[6]; cosi = th[3]
    t = np.linspace(1e7, 2e8, 50)
    # the retarded phase is ~1e4 rad, rounded to ~1e-12 rad: a 1e3 s step keeps
    # that below 1e-8 of the derivative, the truncation (W dt)^2 / 6 below 1e-9
    dt = 1e3
    ds = (dense.cw_signal(th, c, t + dt, d_kpc) - dense.cw_signal(th, c, t - dt, d_kpc)) / (2 * dt)

    def z_earth(tt):
        ph = W * tt + th[1]
        return fp * h0 * (1 + cosi ** 2) * np.cos(ph) + fx * 2 * h0 * cosi * np.sin(ph)

    z = z_earth(t) - z_earth(t - tau)
    assert np.allclose(ds, z, rtol=1e-6, atol=1e-9 * np.abs(z).max())


def test_pulsar_term_geometry_limits():
    """Pulsar perpendicular to the source: tau = d/c exactly.  Pulsar
    towards the source: 1 - n.c vanishes (clamped), no delay, no residual."""
    th = np.array([-8.1, 0.7, 0.3, 0.4, 0.0, 0.0, -13.7])       # source along +x
    t = np.linspace(0.0, 3e8, 40)
    c_perp = np.array([0.0, 0.6, 0.8])
    s = dense.cw_signal(th, c_perp, t, 0.9)
    s_e = dense.cw_signal(th, c_perp, t)
    tau = 0.9 * dense.KPC_LIGHT_S
    assert np.allclose(s, s_e - dense.cw_signal(th, c_perp, t - tau), rtol=0, atol=1e-12 * np.abs(s_e).max())
    c_near = np.array([math.cos(1e-4), math.sin(1e-4), 0.0])    # 1e-4 rad from the source
    s_near = dense.cw_signal(th, c_near, t, 0.9)
    assert np.max(np.abs(s_near)) < 1e-3 * np.max(np.abs(dense.cw_signal(th, c_near, t)))


def test_zero_distance_cancels_the_wave_in_the_filter():
    """d -> 0: the pulsar term cancels the Earth term, so the likelihood is
    that of no signal at all."""
    d = pt_array([90, 60], seed=3)
    th = inputs.make_theta_batch(d, 2, seed=2)
    th[:, 9::3] = 1e-15          # d_p, the third slot of each pulsar
    nosig = inputs.ArrayData(off=d.off, t=d.t, r=d.r, sigma=d.sigma, pos=d.pos, equad=d.equad,
                             p0=d.p0, theta_true=d.theta_true)
    th0 = np.concatenate([th[:, :7]] + [th[:, 7 + 3 * p: 9 + 3 * p] for p in range(2)], axis=1)
    th0[:, 6] = -40.0
    assert np.allclose(kalman.loglik(d, th), kalman.loglik(nosig, th0), rtol=1e-12, atol=0)


@pytest.mark.parametrize("model", ["rw", "ou"])
@pytest.mark.parametrize("seed", [0, 1])
def test_kalman_with_pulsar_term_equals_dense_mvn(model, seed):
    d = pt_array([90, 40, 130], seed=60 + seed, model=model)
    for kind in ("posterior", "prior"):
        th = inputs.make_theta_batch(d, 3, seed=seed, kind=kind)
        assert np.allclose(kalman.loglik(d, th), dense.loglik(d, th), rtol=1e-10, atol=0)


def test_pulsar_filter_lane_form_matches_dense():
    """The phase-lag lane (A, B, Omega, Phi0, sigma^2, EFAC, 0, Omega tau) of
    one pulsar against the dense retarded-time form."""
    rng = np.random.default_rng(21)
    n = 150
    t = np.sort(rng.uniform(0, inputs.T_OBS, n)); t -= t[0]
    sigma = np.full(n, 1e-7)
    p0 = np.array(inputs.P0_DEFAULT)
    th = np.array([-8.0, 1.1, 0.5, 0.3, 0.2, 2.0, -13.2])
    c = inputs.isotropic_positions(rng, 1)[0]
    A, B, W, phi0, D = kalman.cw_project(th, c, with_delay=True)
    d_kpc = 0.7
    r = 3e-7 * rng.standard_normal(n)
    lane = np.array([A, B, W, phi0, 1e-39, 1.1, 0.0, W * d_kpc * dense.KPC_LIGHT_S * D])
    ll = kalman.pulsar_filter(t, r, sigma, 0.0, p0, lane)
    C = dense.ibm_covariance(t, 1e-39, p0, (1.1 * sigma) ** 2)
    res = r - dense.cw_signal(th, c, t, d_kpc)
    L = np.linalg.cholesky(C)
    z = np.linalg.solve(L, res)
    ref = -0.5 * (z @ z + 2 * np.sum(np.log(np.diag(L))) + n * math.log(2 * math.pi))
    assert ll == pytest.approx(ref, rel=1e-10)


def _richardson_fd(f, x, j, h):
    def cd(hh):
        xp = x.copy(); xm = x.copy()
        xp[j] += hh; xm[j] -= hh
        return (f(xp) - f(xm)) / (2 * hh)
    return (4 * cd(h / 2) - cd(h)) / 3


def fd_steps(data):
    """Steps for central differences: the pulsar-term phase W d (1 - n.c)/c is
    thousands of radians, so f, the sky position and d_p need small steps."""
    k = data.n_per_pulsar
    h = np.full(data.dim, 1e-4)
    h[[0, 4, 5]] = 1e-8
    h[7 + k - 1::k] = 1e-8
    return h


@pytest.mark.parametrize("model", ["rw", "ou"])
def test_gradient_with_pulsar_term_vs_finite_differences_and_dense(model):
    d = pt_array([110, 60], seed=71, model=model, equad=1e-8)
    th = inputs.make_theta_batch(d, 1, seed=3)[0]
    _, g = kalman.loglik_grad(d, th)
    f = lambda x: kalman.loglik(d, x)[0]
    h = fd_steps(d)
    fd = np.array([_richardson_fd(f, th, j, h[j]) for j in range(d.dim)])
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert np.max(np.abs(g[0] - fd) / scale) <= 1e-5
    gd = dense.grad(d, th)
    scale = np.maximum(np.abs(gd), 1e-6 * np.abs(gd).max())
    assert np.max(np.abs(g[0] - gd) / scale) <= 1e-7


def test_out_of_domain_distance():
    d = pt_array([40, 30], seed=42, model="ou")
    th = inputs.make_theta_batch(d, 3, seed=7)
    th[0, 10] = 0.0          # d of pulsar 0 (fourth slot)
    th[1, 14] = -0.5         # d of pulsar 1
    ll, g = kalman.loglik_grad(d, th)
    assert np.all(np.isneginf(ll[:2])) and np.isfinite(ll[2])
    assert np.all(g[:2] == 0) and np.all(np.isfinite(g[2]))
