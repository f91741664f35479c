"""Dense (definition-level) oracle: the multivariate-normal log-density of each
pulsar's residual vector.  TEST INFRASTRUCTURE ONLY.

The Kalman filter's prediction-error decomposition reaches this exactly, up to
rounding (paper, Statement of Need and Relation to Existing Work: the
state-space likelihood is the time-domain form of the Gaussian-process
likelihood that frequency-domain methods evaluate with full covariance
matrices).  Here that covariance is written out and factorised by Cholesky,
O(N^3): usable for N up to a few thousand.

Model (paper, Functionality: linear SDEs for the pulsar's spin wandering,
separated from EFAC/EQUAD white measurement noise): with tau = t - t_1,

  C_ij = P0_rr + P0_ry (tau_i + tau_j) + P0_yy tau_i tau_j
         + sigma_p^2 (m^2 M / 2 - m^3 / 6) + delta_ij R_i,
  m = min(tau_i, tau_j),  M = max(tau_i, tau_j),  R_i = EFAC^2 sigma_i^2 + EQUAD^2

(the covariance of a once-integrated Brownian motion plus the propagated
prior), and ll_p = -1/2 [(r - s)^T C^-1 (r - s) + ln det C + N ln 2 pi].

With Ornstein-Uhlenbeck red noise (paper, Functionality: OU processes for
pulsar-intrinsic red noise), dy = -gam y dt + sigma_p dW, so y(tau) =
e^{-gam tau} y_1 + eta(tau) and rho(tau) = rho_1 + g(tau) y_1 + int_0^tau eta,
g(tau) = (1 - e^{-gam tau}) / gam.  Then

  C_ij = P0_rr + P0_ry (g_i + g_j) + P0_yy g_i g_j
         + sigma_p^2 int_0^m g(v) g(v + M - m) dv + delta_ij R_i,

  int_0^m g(v) g(v + d) dv
    = [m - g(m) - e^{-gam d} g(m) + e^{-gam d} (1 - e^{-2 gam m}) / (2 gam)] / gam^2

(the covariance of the integral of an OU process started at zero), which
tends to the integrated-Brownian-motion kernel as gam -> 0.

With the wave's pulsar term the residual is the Earth term minus the same
Earth-term residual at the retarded time t - tau_p, tau_p = d_p (1 - n.c)/c
(d_p the pulsar's distance): s(t) = s_E(t) - s_E(t - tau_p).

Gradients: d ll / d theta = (ds/dtheta)^T alpha for the signal parameters and
1/2 tr[(alpha alpha^T - C^-1) dC/deta] for the noise parameters, with
alpha = C^-1 (r - s).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_factor, cho_solve

LN10 = np.log(10.0)
N_GW = 7
# light-travel time over one kiloparsec, s (IAU: 1 pc = 648000/pi au, au and c exact)
KPC_LIGHT_S = 1e3 * (648000.0 / np.pi) * 149597870700.0 / 299792458.0


def cw_project(theta_gw, pos):
    """(A, B, Omega, Phi0) of the Earth-term continuous-wave residual.

    Works for real or complex theta (complex-step derivatives).
    """
    th = np.asarray(theta_gw)
    f = 10.0 ** th[0]
    W = 2.0 * np.pi * f
    phi0, psi, cosi, sind, al, h0 = th[1], th[2], th[3], th[4], th[5], 10.0 ** th[6]
    cosd = np.sqrt(1.0 - sind * sind)
    n = np.array([cosd * np.cos(al), cosd * np.sin(al), sind])
    u = np.array([np.sin(al), -np.cos(al), 0.0 * al])
    v = np.array([sind * np.cos(al), sind * np.sin(al), -cosd])
    p = np.cos(psi) * u + np.sin(psi) * v
    q = -np.sin(psi) * u + np.cos(psi) * v
    c = np.asarray(pos, dtype=np.float64)
    cp, cq = c @ p, c @ q
    D = 1.0 - c @ n
    if np.real(D) < 1e-12:
        D = 1e-12 + 1j * np.imag(D) if np.iscomplexobj(D) else 1e-12
    Fp = 0.5 * (cp * cp - cq * cq) / D
    Fx = cp * cq / D
    A = Fp * h0 * (1.0 + cosi * cosi) / W
    B = -2.0 * Fx * h0 * cosi / W
    return A, B, W, phi0


def _delay_factor(theta_gw, pos):
    """1 - n.c, clamped as in the antenna pattern."""
    th = np.asarray(theta_gw)
    sind, al = th[4], th[5]
    cosd = np.sqrt(1.0 - sind * sind)
    n = np.array([cosd * np.cos(al), cosd * np.sin(al), sind])
    D = 1.0 - np.asarray(pos, dtype=np.float64) @ n
    if np.real(D) < 1e-12:
        D = 1e-12 + 1j * np.imag(D) if np.iscomplexobj(D) else 1e-12
    return D


def cw_signal(theta_gw, pos, t, d_kpc=None):
    """The continuous-wave residual; with a distance d_kpc, Earth minus pulsar term."""
    A, B, W, phi0 = cw_project(theta_gw, pos)
    t = np.asarray(t)
    s_earth = lambda tt: A * np.sin(W * tt + phi0) + B * np.cos(W * tt + phi0)
    s = s_earth(t)
    if d_kpc is not None:
        tau = d_kpc * KPC_LIGHT_S * _delay_factor(theta_gw, pos)
        s = s - s_earth(t - tau)
    return s


def ibm_covariance(t, sig2, p0, R):
    """Dense covariance of the residual vector of one pulsar."""
    tau = np.asarray(t, dtype=np.float64) - t[0]
    mn = np.minimum.outer(tau, tau)
    mx = np.maximum.outer(tau, tau)
    C = (p0[0] + p0[1] * (tau[:, None] + tau[None, :]) + p0[2] * np.outer(tau, tau)
         + sig2 * (mn * mn * mx / 2.0 - mn ** 3 / 6.0))
    C[np.diag_indices_from(C)] += R
    return C


def ou_covariance(t, sig2, gam, p0, R):
    """Dense covariance of one pulsar's residuals under OU red noise (gam may be
    complex, for complex-step derivatives in gam)."""
    tau = np.asarray(t, dtype=np.float64) - t[0]
    mn = np.minimum.outer(tau, tau)
    d = np.maximum.outer(tau, tau) - mn
    g = -np.expm1(-gam * tau) / gam
    gm = -np.expm1(-gam * mn) / gam
    ed = np.exp(-gam * d)
    K = (mn - gm - ed * gm - ed * np.expm1(-2.0 * gam * mn) / (2.0 * gam)) / (gam * gam)
    C = p0[0] + p0[1] * (g[:, None] + g[None, :]) + p0[2] * np.outer(g, g) + sig2 * K
    C[np.diag_indices_from(C)] += R
    return C


def _layout(data):
    """(parameters per pulsar, OU?, pulsar term?)"""
    ou = getattr(data, "model", "rw") == "ou"
    pt = bool(getattr(data, "pulsar_term", False))
    return 2 + int(ou) + int(pt), ou, pt


def _noise(data, p, theta):
    """(sig2, gam or None, efac, parameters per pulsar, d or None) of pulsar p."""
    k, ou, pt = _layout(data)
    nz = theta[N_GW + k * p:N_GW + k * (p + 1)]
    gam = 10.0 ** nz[1] if ou else None
    efac = nz[2] if ou else nz[1]
    return 10.0 ** (2.0 * nz[0]), gam, efac, k, (nz[-1] if pt else None)


def _pulsar_parts(data, p, theta):
    t, r, sig = data.pulsar(p)
    sig2, gam, efac, _, d = _noise(data, p, theta)
    R = efac ** 2 * sig ** 2 + data.equad[p] ** 2
    if gam is None:
        C = ibm_covariance(t, sig2, data.p0[p], R)
    else:
        C = ou_covariance(t, sig2, gam, data.p0[p], R)
    s = cw_signal(theta[:N_GW], data.pos[p], t, d)
    return t, r, sig, sig2, efac, C, s


def pulsar_loglik(data, p, theta):
    t, r, sig, sig2, efac, C, s = _pulsar_parts(data, p, theta)
    cf = cho_factor(C, lower=True)
    d = r - s
    alpha = cho_solve(cf, d)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    return -0.5 * (d @ alpha + logdet + len(t) * np.log(2.0 * np.pi))


def loglik(data, theta):
    theta = np.atleast_2d(theta)
    return np.array([sum(pulsar_loglik(data, p, th) for p in range(data.n_pulsars))
                     for th in theta])


def grad(data, theta, h=1e-20):
    """Gradient by the dense formulas; ds/dtheta by complex step on cw_signal."""
    theta = np.asarray(theta, dtype=np.float64)
    P = data.n_pulsars
    k, ou, pt = _layout(data)
    g = np.zeros(N_GW + k * P)
    for p in range(P):
        t, r, sig, sig2, efac, C, s = _pulsar_parts(data, p, theta)
        d = theta[N_GW + k * p + k - 1] if pt else None
        cf = cho_factor(C, lower=True)
        alpha = cho_solve(cf, r - s)
        for j in range(N_GW):
            thc = theta[:N_GW].astype(np.complex128)
            thc[j] += 1j * h
            ds = np.imag(cw_signal(thc, data.pos[p], t, d)) / h
            g[j] += ds @ alpha
        if pt:
            ds = np.imag(cw_signal(theta[:N_GW], data.pos[p], t, d + 1j * h)) / h
            g[N_GW + k * p + k - 1] = ds @ alpha
        Cinv = cho_solve(cf, np.eye(len(t)))
        M = np.outer(alpha, alpha) - Cinv
        R = efac ** 2 * sig ** 2 + data.equad[p] ** 2
        if not ou:
            tau = t - t[0]
            mn = np.minimum.outer(tau, tau)
            mx = np.maximum.outer(tau, tau)
            dC_ls = 2.0 * LN10 * sig2 * (mn * mn * mx / 2.0 - mn ** 3 / 6.0)
        else:
            # the red-noise part is proportional to sigma_p^2
            lg = theta[N_GW + k * p + 1]
            zero = np.zeros(3)
            dC_ls = 2.0 * LN10 * (ou_covariance(t, sig2, 10.0 ** lg, zero, 0.0))
            thc = 10.0 ** (lg + 1j * h)
            dC_lg = np.imag(ou_covariance(t, sig2, thc, data.p0[p], R)) / h
            g[N_GW + k * p + 1] = 0.5 * np.sum(M * dC_lg)
        g[N_GW + k * p] = 0.5 * np.sum(M * dC_ls)
        g[N_GW + k * p + (2 if ou else 1)] = 0.5 * np.sum(np.diag(M) * 2.0 * efac * sig ** 2)
    return g


# ---------------------------------------------------------------------------
# Joint likelihood with a Hellings-Downs correlated GW background (the model
# stated in gwb_body.h): per pulsar rho integrates its own OU red noise y and
# the GW redshift a; the a_n are stationary OU processes (damping gamma_a)
# whose driving noises are correlated across pulsars by the HD matrix G, with
# amplitude h_a.  The residual covariance, all TOAs of all pulsars, is
#   C = blockdiag_n(C_int,n + R_n) + h_a^2 (G_nm K(t_i, t_j))_{(n,i),(m,j)},
# C_int,n the OU-integrated covariance from the prior P0_n at the array's
# earliest TOA t_0, and K the covariance of the time integrals from t_0 of a
# stationary unit-noise OU process:
#   K(u, v) = int_0^u int_0^v e^{-gamma |s - s'|} ds ds' / (2 gamma)
#           = [2 E(gamma m) + g(gamma m) g(gamma |u - v|)] / (2 gamma^3),
#   m = min(u, v),  g(x) = 1 - e^-x,  E(x) = x - g(x)   (both terms >= 0).
# ---------------------------------------------------------------------------
def hellings_downs(pos):
    pos = np.asarray(pos, dtype=np.float64)
    c = np.clip(pos @ pos.T, -1.0, 1.0)
    x = 0.5 * (1.0 - c)
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.where(x > 0, 1.5 * x * np.log(np.where(x > 0, x, 1.0)), 0.0) - 0.25 * x + 0.5
    np.fill_diagonal(G, 1.0)
    return G


def _E(x):
    """x - (1 - e^-x), without cancellation."""
    x = np.asarray(x, dtype=np.float64)
    small = x < 0.1
    xs = np.where(small, x, 0.0)
    ser = np.zeros_like(x)
    term = xs * xs / 2.0
    for k in range(2, 20):
        ser = ser + term
        term = -term * xs / (k + 1)
    return np.where(small, ser, x + np.expm1(-np.where(small, 1.0, x)))


def gw_integrated_kernel(u, v, gam):
    """K(u, v) for arrays u [n], v [m] (seconds since t_0)."""
    u = np.asarray(u, dtype=np.float64)[:, None]
    v = np.asarray(v, dtype=np.float64)[None, :]
    mn = np.minimum(u, v)
    d = np.abs(u - v)
    g = lambda z: -np.expm1(-z)
    return (2.0 * _E(gam * mn) + g(gam * mn) * g(gam * d)) / (2.0 * gam ** 3)


def gwb_covariance(data, theta):
    P = data.n_pulsars
    t0 = data.t.min() if len(data.t) else 0.0
    G = hellings_downs(data.pos)
    ha2, ga = 10.0 ** (2.0 * theta[0]), 10.0 ** theta[1]
    blocks = []
    for p in range(P):
        t, r, sig = data.pulsar(p)
        ls, lg, efac = theta[2 + 3 * p: 5 + 3 * p]
        R = efac ** 2 * sig ** 2 + data.equad[p] ** 2
        Ci = ou_covariance(np.concatenate([[t0], t]), 10.0 ** (2 * ls), 10.0 ** lg, data.p0[p], 0.0)[1:, 1:]
        blocks.append(Ci + np.diag(R))
    n = len(data.t)
    C = np.zeros((n, n))
    for a in range(P):
        ta = data.pulsar(a)[0] - t0
        sa = slice(data.off[a], data.off[a + 1])
        C[sa, sa] += blocks[a]
        for b in range(P):
            tb = data.pulsar(b)[0] - t0
            sb = slice(data.off[b], data.off[b + 1])
            C[sa, sb] += ha2 * G[a, b] * gw_integrated_kernel(ta, tb, ga)
    return C


def gwb_loglik(data, theta):
    theta = np.atleast_2d(theta)
    out = []
    for th in theta:
        C = gwb_covariance(data, th)
        cf = cho_factor(C, lower=True)
        alpha = cho_solve(cf, data.r)
        logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
        out.append(-0.5 * (data.r @ alpha + logdet + len(data.r) * np.log(2.0 * np.pi)))
    return np.array(out)
