"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index, a
transposed operand) in a private copy of the C oracle, compiles it on the CPU,
and checks that at least one pin fails; the unmodified copy must pass all of
them.
"""
from __future__ import annotations

import math
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import dense, exact, kalman
from paper_2510_11077_gb300 import inputs

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTATIONS = {
    "drop_q01": ("kf_body.h", "KF_T a01 = a * (p01 + b * p11) + q01;", "KF_T a01 = a * (p01 + b * p11);"),
    "q00_factor": ("kf_body.h", "dt * dt * dt / 3.0", "dt * dt * dt / 2.0"),
    "innovation_sign": ("kf_body.h", "r[k] - s - mp0", "r[k] - s + mp0"),
    "gain_transposed": ("kf_body.h", "K0 = a00 / S, K1 = a01 / S", "K0 = a01 / S, K1 = a00 / S"),
    "p11_index": ("kf_body.h", "p11 = a11 - K1 * S * K1", "p11 = a11 - K0 * S * K1"),
    "p01_index": ("kf_body.h", "p01 = a01 - K0 * S * K1", "p01 = a01 - K0 * S * K0"),
    "drop_log2pi": ("kf_body.h", "KF_LOG2PI + KF_LOG(S)", "KF_LOG(S)"),
    "mean_predict": ("kf_body.h", "KF_T mp0 = m0 + b * m1;", "KF_T mp0 = m0;"),
    "a00_cross_term": ("kf_body.h", "p00 + b * p01 + b * p01", "p00 + b * p01"),
    "efac_not_squared": ("kf_body.h", "efac * efac * (sigma[k] * sigma[k])", "efac * (sigma[k] * sigma[k])"),
    "dt_from_first": ("kf_body.h", "t[k] - t[k - 1]", "t[k] - t[0]"),
    "phase_sign": ("kf_body.h", "Om * t[k] + Phi0", "Om * t[k] - Phi0"),
    "sin_cos_swapped": ("kf_body.h", "A * KF_SIN(phase) + B * KF_COS(phase)",
                        "A * KF_COS(phase) + B * KF_SIN(phase)"),
    "B_sign": ("kalman.c", "*B = -2.0 * Fx", "*B = 2.0 * Fx"),
    "Fplus_half": ("kalman.c", "cplx Fp = 0.5 * (cp * cp - cq * cq) / D;", "cplx Fp = (cp * cp - cq * cq) / D;"),
    "q_basis_sign": ("kalman.c", "q[i] = -csin(psi) * u[i]", "q[i] = csin(psi) * u[i]"),
    "v_basis_sign": ("kalman.c", "sind * csin(al), -cosd}", "sind * csin(al), cosd}"),
    "h0_index": ("kalman.c", "cplx h0 = cpow(10.0, th[6]);", "cplx h0 = cpow(10.0, th[5]);"),
    "noise_grads_swapped": ("kalman.c", "g[N_GW + np * p + i] = cimag(lp) / CS_H;",
                            "g[N_GW + np * p + (i + 1) % np] = cimag(lp) / CS_H;"),
    "omega_no_2pi": ("kalman.c", "cplx W = 2.0 * M_PI * f;", "cplx W = M_PI * f;"),
    # Ornstein-Uhlenbeck red noise
    "ou_decay_first_order": ("kf_body.h", "a = 1.0 - gam * dt * p1;", "a = 1.0 - gam * dt;"),
    "ou_q01_phi": ("kf_body.h", "q01 = q01 * p1 * p1;", "q01 = q01 * p1;"),
    "ou_q11_phi": ("kf_body.h", "q11 = q11 * p2;", "q11 = q11 * p1;"),
    "ou_a01_no_decay": ("kf_body.h", "KF_T a01 = a * (p01 + b * p11) + q01;", "KF_T a01 = p01 + b * p11 + q01;"),
    "ou_a11_decay_once": ("kf_body.h", "KF_T a11 = a * a * p11 + q11;", "KF_T a11 = a * p11 + q11;"),
    "ou_phi4_series": ("ou_phi.h", "(2.0 - pow(2.0, m + 2))", "(2.0 - pow(2.0, m + 1))"),
    "ou_phi1_series_sign": ("ou_phi.h", "double c1 = ((m & 1) ? -1.0 : 1.0) / f1;", "double c1 = 1.0 / f1;"),
    "ou_phi2_closed": ("ou_phi.h", "*p2 = (1.0 - e2) / (2.0 * x);", "*p2 = (1.0 - e2) / x;"),
    "ou_phi4_closed": ("ou_phi.h", "0.5 * (1.0 - e2)) / (x * x * x)", "(1.0 - e2)) / (x * x * x)"),
    "ou_gamma_index": ("kalman.c", "cplx gam = a->ou ? cpow(10.0, nz[1]) : 0.0;",
                       "cplx gam = a->ou ? cpow(10.0, nz[0]) : 0.0;"),
    # the wave's pulsar term
    "pt_sign": ("kf_body.h", "if (pt) s -= A", "if (pt) s += A"),
    "pt_lag_sign": ("kf_body.h", "KF_SIN(phase - Dp) + B * KF_COS(phase - Dp)",
                    "KF_SIN(phase + Dp) + B * KF_COS(phase + Dp)"),
    "pt_no_geometry": ("kalman.c", "Om * (nz[n_noise(a) - 1] * KPC_LIGHT_S * Dn)",
                       "Om * (nz[n_noise(a) - 1] * KPC_LIGHT_S)"),
    "pt_light_speed_km": ("kalman.c", "149597870700.0 / 299792458.0)", "149597870700.0 / 299792.458)"),
    "pt_efac_slot": ("kalman.c", "static int efac_slot(const array_view* a) { return 1 + a->ou; }",
                     "static int efac_slot(const array_view* a) { return n_noise(a) - 1; }"),
    "pt_real_distance_index": ("kalman.c", "creal(Om) * (nz[np - 1] * KPC_LIGHT_S",
                               "creal(Om) * (nz[np - 2] * KPC_LIGHT_S"),
}


def _build_variant(tmp, name, mut):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    for f in ("kalman.c", "kf_body.h", "ou_phi.h"):
        shutil.copy(os.path.join(ORACLE_DIR, f), d)
    if mut is not None:
        fname, old, new = mut
        path = os.path.join(d, fname)
        src = open(path).read()
        assert src.count(old) == 1, (name, old)
        open(path, "w").write(src.replace(old, new))
    lib = os.path.join(d, "lib.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-D_GNU_SOURCE", "-o", lib,
                    os.path.join(d, "kalman.c"), "-lm"], check=True)
    return lib


def _pins(lib):
    """Fast versions of the pins; returns the names of those that fail."""
    failed = []
    d = inputs.make_array(np.array([80, 33]), seed=3, equad=2e-8)
    th = inputs.make_theta_batch(d, 1, seed=1)[0]
    th[7::2] = -19.3
    # dense multivariate normal
    ll = kalman.loglik(d, th, lib_path=lib)[0]
    ref = dense.loglik(d, th)[0]
    if not abs(ll - ref) <= 1e-10 * abs(ref):
        failed.append("dense")
    # exact rational brute force, no signal
    t = np.array([0.0, 1e6, 4e6, 2e7]); r = np.array([1e-7, 3e-7, -2e-7, 5e-8])
    sigma = np.full(4, 1e-7); p0 = np.array([1e-14, 1e-24, 1e-32])
    lane = np.array([0.0, 0.0, 1e-8, 0.0, 1e-38, 0.9])
    ll = kalman.pulsar_filter(t, r, sigma, 0.0, p0, lane, lib_path=lib)
    C = exact.covariance([Fr(x) for x in t], Fr(1e-38), [Fr(x) for x in p0],
                         [Fr(0.9) ** 2 * Fr(1e-7) ** 2] * 4)
    det, quad = exact.det_and_quad(C, [Fr(x) for x in r])
    ll_ex = -0.5 * (float(quad) + math.log(det.numerator) - math.log(det.denominator)
                    + 4 * math.log(2 * math.pi))
    if not abs(ll - ll_ex) <= 1e-12 * abs(ll_ex):
        failed.append("exact")
    # gradient against central differences of the same library's value
    _, g = kalman.loglik_grad(d, th, lib_path=lib)
    f = lambda x: kalman.loglik(d, x, lib_path=lib)[0]
    fd = []
    for j in range(d.dim):
        h = 1e-7 if j == 0 else 1e-4
        xp, xm = th.copy(), th.copy(); xp[j] += h; xm[j] -= h
        fd.append((f(xp) - f(xm)) / (2 * h))
    fd = np.array(fd)
    if not np.all(np.abs(g[0] - fd) <= 1e-4 * np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())):
        failed.append("fd")
    # Ornstein-Uhlenbeck red noise: dense likelihood (steps on both sides of
    # the series / closed-form switch) and the dense gradient
    rng = np.random.default_rng(3)
    tt = np.cumsum(np.concatenate([rng.uniform(1e5, 4e6, 25), rng.uniform(5e6, 3e7, 20)]))
    do = inputs.ArrayData(off=np.array([0, 45]), t=tt, r=1e-6 * rng.standard_normal(45),
                          sigma=np.full(45, 1e-7), pos=np.array([[0.6, 0.0, 0.8]]),
                          equad=np.array([1e-8]), p0=np.array([inputs.P0_DEFAULT]),
                          theta_true=np.zeros(10), model="ou")
    tho = np.array([-8.3, 0.5, 0.4, 0.2, 0.1, 1.0, -13.5, -19.5, -7.0, 1.05])
    llo = kalman.loglik(do, tho, lib_path=lib)[0]
    if not abs(llo - dense.loglik(do, tho)[0]) <= 1e-10 * abs(llo):
        failed.append("dense_ou")
    _, go = kalman.loglik_grad(do, tho, lib_path=lib)
    gd = dense.grad(do, tho)
    if not np.all(np.abs(go[0] - gd) <= 1e-6 * np.maximum(np.abs(gd), 1e-3 * np.abs(gd).max())):
        failed.append("grad_ou")
    # the wave's pulsar term with OU red noise: dense likelihood and gradient
    dp = inputs.make_array(np.array([70, 45]), seed=5, equad=1e-8, model="ou", pulsar_term=True)
    thp = inputs.make_theta_batch(dp, 1, seed=2)[0]
    llp = kalman.loglik(dp, thp, lib_path=lib)[0]
    if not abs(llp - dense.loglik(dp, thp)[0]) <= 1e-10 * abs(llp):
        failed.append("dense_pt")
    _, gp = kalman.loglik_grad(dp, thp, lib_path=lib)
    gdp = dense.grad(dp, thp)
    if not np.all(np.abs(gp[0] - gdp) <= 1e-6 * np.maximum(np.abs(gdp), 1e-3 * np.abs(gdp).max())):
        failed.append("grad_pt")
    # antenna pattern: textbook case (source at the pole, pulsar on the equator)
    thp = np.array([-8.0, 0.0, 0.0, 0.5, 1.0, 0.0, -14.0])
    A, B, W, _ = kalman.cw_project(thp, np.array([1.0, 0.0, 0.0]), lib_path=lib)
    fp = A * W / (1e-14 * 1.25)
    if not abs(abs(fp) - 0.5) < 1e-12:
        failed.append("textbook")
    return failed


@pytest.fixture(scope="module")
def tmpdir_mod(tmp_path_factory):
    return str(tmp_path_factory.mktemp("oracle_mutants"))


def test_unmodified_copy_passes_all_pins(tmpdir_mod):
    lib = _build_variant(tmpdir_mod, "control", None)
    assert _pins(lib) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmpdir_mod, name):
    lib = _build_variant(tmpdir_mod, name, MUTATIONS[name])
    with np.errstate(all="ignore"):
        failed = _pins(lib)
    assert failed, f"mutation {name} passed every pin"
