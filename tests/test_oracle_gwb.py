"""Pins of the joint-likelihood oracle with a Hellings-Downs correlated GW
background (the model stated in oracle/gwb_body.h).

The joint Kalman filter (all TOAs of all pulsars in time order) and the dense
covariance (closed-form kernels) are two formulations of one model; the pins
tie them to each other and to things fixed outside both: the Hellings-Downs
curve as the sky average of the project's antenna patterns, the integrated
OU kernel by quadrature and by simulating the process, the h_a -> 0 limit
(independent OU pulsars, pinned on their own), finite differences, and
planted mistakes.
"""
from __future__ import annotations

import math
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import integrate

from oracle import dense, gwb, kalman
from paper_2510_11077_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def gwb_theta(P, rng, lh=-19.3, lg=-8.2):
    nz = np.stack([rng.uniform(-20.5, -19.5, P), rng.uniform(-9.5, -7.5, P), rng.uniform(0.9, 1.1, P)], 1)
    return np.concatenate([[lh, lg], nz.ravel()])


def _antenna_many(c, n_src, psi):
    """F+, Fx of pulsar direction c for many source directions n_src [M, 3]
    and polarisation angles psi [M] (the definitions of the CW projection)."""
    sind = n_src[:, 2]
    cosd = np.sqrt(1 - sind ** 2)
    al = np.arctan2(n_src[:, 1], n_src[:, 0])
    u = np.stack([np.sin(al), -np.cos(al), np.zeros_like(al)], 1)
    v = np.stack([sind * np.cos(al), sind * np.sin(al), -cosd], 1)
    p = np.cos(psi)[:, None] * u + np.sin(psi)[:, None] * v
    q = -np.sin(psi)[:, None] * u + np.cos(psi)[:, None] * v
    D = 1 - n_src @ c
    cp, cq = p @ c, q @ c
    return 0.5 * (cp ** 2 - cq ** 2) / D, cp * cq / D


@pytest.mark.parametrize("theta_deg", [10.0, 49.0, 82.0, 120.0, 170.0])
def test_hellings_downs_is_the_sky_average_of_antenna_products(theta_deg):
    """G(theta) = (3/2) < F+_a F+_b + Fx_a Fx_b > over isotropic, unpolarised
    sources, which the n -> m limit normalises to 1/2."""
    rng = np.random.default_rng(int(theta_deg))
    M = 400_000
    z = rng.uniform(-1, 1, M); ph = rng.uniform(0, 2 * np.pi, M)
    n_src = np.stack([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z], 1)
    psi = rng.uniform(0, np.pi, M)
    th = math.radians(theta_deg)
    ca = np.array([0.0, 0.0, 1.0]); cb = np.array([math.sin(th), 0.0, math.cos(th)])
    fpa, fxa = _antenna_many(ca, n_src, psi)
    fpb, fxb = _antenna_many(cb, n_src, psi)
    prod = 1.5 * (fpa * fpb + fxa * fxb)
    mc, se = prod.mean(), prod.std() / math.sqrt(M)
    G = gwb.hellings_downs(np.stack([ca, cb]))[0, 1]
    assert abs(G - mc) < 5 * se + 2e-3, (G, mc, se)


def test_hellings_downs_special_values_and_c_numpy_agreement():
    pos = np.array([[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, 1e-5, 1.0 - 5e-11]])
    pos /= np.linalg.norm(pos, axis=1, keepdims=True)
    G = gwb.hellings_downs(pos)
    assert G[0, 1] == pytest.approx(0.25, abs=1e-14)                     # antipodal
    assert G[0, 2] == pytest.approx(0.75 * math.log(0.5) - 0.125 + 0.5, abs=1e-14)   # 90 deg
    assert G[0, 3] == pytest.approx(0.5, abs=1e-8)                       # co-located, distinct
    assert np.all(np.diag(G) == 1.0) and np.allclose(G, G.T)
    rng = np.random.default_rng(3)
    q = inputs.isotropic_positions(rng, 12)
    assert np.allclose(gwb.hellings_downs(q), dense.hellings_downs(q), rtol=0, atol=1e-14)


def test_hd_matrix_is_positive_definite_for_random_arrays():
    rng = np.random.default_rng(8)
    for P in (5, 20, 67):
        G = gwb.hellings_downs(inputs.isotropic_positions(rng, P))
        assert np.linalg.eigvalsh(G).min() > 0.0


@pytest.mark.parametrize("gam", [1e-9, 3e-8])
def test_integrated_ou_kernel_vs_quadrature(gam):
    rng = np.random.default_rng(int(gam * 1e10))
    u = np.sort(rng.uniform(0, inputs.T_OBS, 4))
    K = dense.gw_integrated_kernel(u, u, gam)
    def inner(s1, hi):
        # split at the kink s2 = s1 of |s1 - s2|
        f = lambda s2: math.exp(-gam * abs(s1 - s2)) / (2 * gam)
        cut = min(max(s1, 0.0), hi)
        a = integrate.quad(f, 0.0, cut, epsabs=0, epsrel=1e-12, limit=200)[0] if cut > 0 else 0.0
        b = integrate.quad(f, cut, hi, epsabs=0, epsrel=1e-12, limit=200)[0] if hi > cut else 0.0
        return a + b

    for i in range(4):
        for j in range(i, 4):
            val = integrate.quad(lambda s1: inner(s1, u[j]), 0.0, u[i], epsabs=0, epsrel=1e-10,
                                 limit=200, points=[u[j]] if u[j] < u[i] else None)[0]
            assert K[i, j] == pytest.approx(val, rel=1e-7)


def test_integrated_ou_kernel_vs_simulated_process():
    """Stationary unit-noise OU (exact AR(1) steps), integrated by the
    trapezoid rule: the empirical covariance of the integrals."""
    rng = np.random.default_rng(4)
    gam, T, steps, paths = 1.0, 3.0, 600, 40_000
    h = T / steps
    a = rng.standard_normal(paths) * math.sqrt(1 / (2 * gam))
    I = np.zeros(paths)
    keep = {150: None, 400: None, 600: None}
    hist = {}
    phi = math.exp(-gam * h); sd = math.sqrt((1 - phi * phi) / (2 * gam))
    for k in range(1, steps + 1):
        a_new = phi * a + sd * rng.standard_normal(paths)
        I += 0.5 * h * (a + a_new)
        a = a_new
        if k in keep:
            hist[k] = I.copy()
    ts = np.array(sorted(keep)) * h
    emp = np.cov(np.stack([hist[k] for k in sorted(keep)]))
    K = dense.gw_integrated_kernel(ts, ts, gam)
    assert np.allclose(emp, K, rtol=0.05, atol=0.02 * K.max())


@pytest.mark.parametrize("seed,lh,lg", [(0, -19.3, -8.2), (1, -18.5, -9.6), (2, -19.0, -7.1), (3, -20.5, -10.0)])
def test_joint_kalman_equals_dense_mvn(seed, lh, lg):
    rng = np.random.default_rng(seed)
    d = inputs.make_array(np.array([45, 20, 70]), seed=100 + seed, equad=1e-8)
    th = gwb_theta(3, rng, lh, lg)
    assert gwb.loglik(d, th)[0] == pytest.approx(dense.gwb_loglik(d, th)[0], rel=1e-10)


def test_equal_times_across_pulsars_and_empty_pulsar():
    rng = np.random.default_rng(7)
    d = inputs.make_array(np.array([30, 0, 25]), seed=7)
    # pulsar 2 shares five TOA times with pulsar 0
    d.t[d.off[2]:d.off[2] + 5] = d.t[d.off[0] + 3:d.off[0] + 8]
    d.t[d.off[2]:d.off[3]] = np.sort(d.t[d.off[2]:d.off[3]])
    th = gwb_theta(3, rng)
    assert gwb.loglik(d, th)[0] == pytest.approx(dense.gwb_loglik(d, th)[0], rel=1e-10)


def test_vanishing_background_gives_independent_ou_pulsars():
    """h_a -> 0 with every pulsar's first TOA at the array epoch: the joint
    likelihood is the sum of the per-pulsar OU likelihoods (no CW source)."""
    rng = np.random.default_rng(9)
    d = inputs.make_array(np.array([40, 55, 30]), seed=9, model="ou")
    for p in range(3):
        d.t[d.off[p]] = 0.0
    th = gwb_theta(3, rng, lh=-40.0)
    th_ou = np.concatenate([[-8.0, 0.3, 0.2, 0.1, 0.4, 1.0, -40.0], th[2:]])
    assert gwb.loglik(d, th)[0] == pytest.approx(kalman.loglik(d, th_ou)[0], rel=1e-12)


def test_pulsar_order_does_not_matter():
    rng = np.random.default_rng(11)
    d = inputs.make_array(np.array([30, 45, 20]), seed=11)
    th = gwb_theta(3, rng)
    perm = [2, 0, 1]
    d2 = inputs.ArrayData(off=np.concatenate([[0], np.cumsum(d.n_toa[perm])]),
                          t=np.concatenate([d.pulsar(p)[0] for p in perm]),
                          r=np.concatenate([d.pulsar(p)[1] for p in perm]),
                          sigma=np.concatenate([d.pulsar(p)[2] for p in perm]),
                          pos=d.pos[perm], equad=d.equad[perm], p0=d.p0[perm], theta_true=d.theta_true)
    th2 = np.concatenate([th[:2]] + [th[2 + 3 * p: 5 + 3 * p] for p in perm])
    assert gwb.loglik(d2, th2)[0] == pytest.approx(gwb.loglik(d, th)[0], rel=1e-12)


def test_gradient_vs_richardson_finite_differences():
    rng = np.random.default_rng(13)
    d = inputs.make_array(np.array([40, 30]), seed=13, equad=1e-8)
    th = gwb_theta(2, rng, lh=-18.8, lg=-8.0)
    _, g = gwb.loglik_grad(d, th)
    f = lambda x: gwb.loglik(d, x)[0]

    def cd(j, h):
        xp, xm = th.copy(), th.copy(); xp[j] += h; xm[j] -= h
        return (f(xp) - f(xm)) / (2 * h)

    fd = np.array([(4 * cd(j, 5e-5) - cd(j, 1e-4)) / 3 for j in range(len(th))])
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert np.max(np.abs(g[0] - fd) / scale) <= 1e-5


def test_out_of_domain():
    rng = np.random.default_rng(14)
    d = inputs.make_array(np.array([20, 20]), seed=14)
    th = np.stack([gwb_theta(2, rng) for _ in range(3)])
    th[0, 4] = 0.0          # EFAC of pulsar 0
    th[1, 1] = np.nan
    ll = gwb.loglik(d, th)
    assert np.all(np.isneginf(ll[:2])) and np.isfinite(ll[2])


MUTATIONS = {
    "hd_autocorrelation_half": ("gwb.c", "if (a == b) { G[a * P + b] = 1.0; continue; }",
                                "if (a == b) { G[a * P + b] = 0.5; continue; }"),
    "hd_log_sign": ("gwb.c", "1.5 * x * log(x)", "-1.5 * x * log(x)"),
    "stationary_prior_no_half": ("gwb_body.h", "ha2 * G[a * P + b] / (2.0 * ga)", "ha2 * G[a * P + b] / ga"),
    "gw_not_in_residual": ("gwb_body.h", "F[R0 * n + A] = ba;", "F[R0 * n + A] = 0.0;"),
    "gw_cross_noise_dropped": ("gwb_body.h", "Q[R0 * n + Ab] += Gab * qa01;", "Q[R0 * n + Ab] += 0.0;"),
    "gw_decay_uses_pulsar_gamma": ("gwb_body.h", "KF_PHI(ga * dt, &a1, &a2, &a4);", "KF_PHI(gp[0] * dt, &a1, &a2, &a4);"),
    "measures_wrong_pulsar": ("gwb_body.h", "const int i0 = 3 * q;", "const int i0 = 3 * (P - 1 - q);"),
}


def _variant(tmp, name, mut):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    for f in ("kalman.c", "kf_body.h", "ou_phi.h", "gwb.c", "gwb_body.h"):
        shutil.copy(os.path.join(ORACLE_DIR, f), d)
    if mut is not None:
        fname, old, new = mut
        path = os.path.join(d, fname)
        src = open(path).read()
        assert src.count(old) == 1, (name, old)
        open(path, "w").write(src.replace(old, new))
    lib = os.path.join(d, "lib.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-D_GNU_SOURCE", "-o", lib,
                    os.path.join(d, "kalman.c"), os.path.join(d, "gwb.c"), "-lm"], check=True)
    return lib


def _gwb_pins(lib):
    failed = []
    rng = np.random.default_rng(21)
    d = inputs.make_array(np.array([35, 25, 40]), seed=21, equad=1e-8)
    th = gwb_theta(3, rng, lh=-18.7, lg=-8.4)
    if not abs(gwb.loglik(d, th, lib_path=lib)[0] - dense.gwb_loglik(d, th)[0]) <= 1e-10 * abs(dense.gwb_loglik(d, th)[0]):
        failed.append("dense")
    q = inputs.isotropic_positions(np.random.default_rng(3), 6)
    if not np.allclose(gwb.hellings_downs(q, lib_path=lib), dense.hellings_downs(q), atol=1e-12):
        failed.append("hd")
    return failed


@pytest.fixture(scope="module")
def tmp_mut(tmp_path_factory):
    return str(tmp_path_factory.mktemp("gwb_mutants"))


def test_unmodified_gwb_copy_passes(tmp_mut):
    assert _gwb_pins(_variant(tmp_mut, "control", None)) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_gwb_mistake_is_caught(tmp_mut, name):
    with np.errstate(all="ignore"):
        assert _gwb_pins(_variant(tmp_mut, name, MUTATIONS[name])), name
