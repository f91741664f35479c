"""Seeded synthetic pulsar-timing-array inputs.

This module only draws random numbers and lays them out; it holds none of the
likelihood's arithmetic (no Kalman step, no gravitational-wave projection).
Both the CPU oracle (tests) and the CUDA path consume what it returns.

Workloads (the arrays the paper's method is meant for: Summary and
Functionality sections; the continuous-wave source of Future Directions):

* ``psr1_toa1000``   1 pulsar, 1000 TOAs, 1 parameter vector
* ``psr20_toa500-2000_w4096``  20 pulsars, 500..2000 TOAs each, 4096 walkers
* ``psr67_toa5000_w1024``      67 pulsars, 5000 TOAs each, 1024 walkers
* ``psr100_toalognormal_w16384`` 100 pulsars, log-normal TOA counts
  (median 3000, sigma_ln 0.8, clipped to [200, 20000]), 16384 walkers

Every TOA set spans 10 years, sorted uniform, TOA error 1e-7 s.  Residuals are
white noise (sigma * EFAC), plus an integrated random walk in fractional
frequency drawn step by step (trapezoidal integration of the phase), plus one
sinusoid per pulsar whose frequency is shared by the array (a generic stand-in
for a continuous gravitational wave: random per-pulsar amplitude and phase).
They carry the value distributions of real timing residuals; the likelihood
does not assume they were drawn from its own model.

Parameter vector layout (D = 7 + 2P for the random-walk red noise):
``[log10 f_gw, Phi0, psi, cos iota, sin delta, alpha, log10 h0,
   (log10 sigma_p, EFAC_p) for p in 0..P-1]``; with Ornstein-Uhlenbeck red
noise (model "ou") each pulsar has ``(log10 sigma_p, log10 gamma_p, EFAC_p)``
and D = 7 + 3P.  With the wave's pulsar term (``pulsar_term=True``) each
pulsar's block ends with its distance d_p in kpc.
"""
from __future__ import annotations

import dataclasses
import numpy as np

YEAR_S = 365.25 * 86400.0
T_OBS = 10.0 * YEAR_S           # 3.15576e8 s
SIGMA_TOA = 1e-7                # s
P0_DEFAULT = (1e-7 ** 2, 0.0, 1e-16 ** 2)   # prior covariance of (rho, y)
N_GW = 7
SEED_BASE = 20251013

# prior box of each parameter (uniform in these coordinates)
PRIOR_GW = np.array([
    [-9.0, -7.0],            # log10 f_gw [Hz]
    [0.0, 2.0 * np.pi],      # Phi0
    [0.0, np.pi],            # psi
    [-1.0, 1.0],             # cos iota
    [-1.0, 1.0],             # sin delta
    [0.0, 2.0 * np.pi],      # alpha
    [-15.0, -13.0],          # log10 h0
])
PRIOR_NOISE = np.array([
    [-21.0, -19.0],          # log10 sigma_p [s^-1/2]
    [0.8, 1.2],              # EFAC
])
PRIOR_NOISE_OU = np.array([
    [-21.0, -19.0],          # log10 sigma_p [s^-1/2]
    [-10.0, -7.0],           # log10 gamma_p [s^-1] (mean reversion 0.3 - 300 yr)
    [0.8, 1.2],              # EFAC
])


PRIOR_DIST = np.array([[0.2, 3.0]])   # pulsar distance d_p [kpc]


def noise_prior(model: str, pulsar_term: bool = False) -> np.ndarray:
    """Prior box of one pulsar's own parameters, in theta order."""
    pr = PRIOR_NOISE_OU if model == "ou" else PRIOR_NOISE
    return np.concatenate([pr, PRIOR_DIST]) if pulsar_term else pr


@dataclasses.dataclass
class ArrayData:
    """A pulsar array in CSR form (pulsar p owns TOAs off[p]:off[p+1])."""
    off: np.ndarray      # int64 [P+1]
    t: np.ndarray        # float64 [sum N], s from the array epoch, sorted per pulsar
    r: np.ndarray        # float64 [sum N], residuals, s
    sigma: np.ndarray    # float64 [sum N], TOA errors, s
    pos: np.ndarray      # float64 [P, 3], unit vectors
    equad: np.ndarray    # float64 [P], s
    p0: np.ndarray       # float64 [P, 3], prior covariance (rr, ry, yy)
    theta_true: np.ndarray  # float64 [D], parameters used to draw the residuals
    model: str = "rw"    # red noise: "rw" random walk, "ou" Ornstein-Uhlenbeck
    pulsar_term: bool = False   # the wave's pulsar term (distance d_p per pulsar)

    @property
    def n_pulsars(self) -> int:
        return len(self.off) - 1

    @property
    def n_noise(self) -> int:
        return 3 if self.model == "ou" else 2

    @property
    def n_per_pulsar(self) -> int:
        """Parameters per pulsar: the noise parameters, then d_p with the pulsar term."""
        return self.n_noise + (1 if self.pulsar_term else 0)

    @property
    def efac_slot(self) -> int:
        return self.n_noise - 1

    @property
    def dim(self) -> int:
        return N_GW + self.n_per_pulsar * self.n_pulsars

    @property
    def n_toa(self) -> np.ndarray:
        return np.diff(self.off)

    def pulsar(self, p: int):
        a, b = self.off[p], self.off[p + 1]
        return self.t[a:b], self.r[a:b], self.sigma[a:b]


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_pulsars: int
    toa_law: tuple           # ("fixed", N) | ("uniform", lo, hi) | ("lognormal", median, s, lo, hi)
    batch: int
    seed: int
    with_signal: bool = True
    grad: bool = True


WORKLOADS = {
    "psr1_toa1000": Workload("psr1_toa1000", 1, ("fixed", 1000), 1, SEED_BASE + 0,
                             with_signal=False, grad=False),
    "psr20_toa500-2000_w4096": Workload("psr20_toa500-2000_w4096", 20, ("uniform", 500, 2000),
                                        4096, SEED_BASE + 1, grad=False),
    "psr67_toa5000_w1024": Workload("psr67_toa5000_w1024", 67, ("fixed", 5000), 1024,
                                    SEED_BASE + 2),
    "psr100_toalognormal_w16384": Workload("psr100_toalognormal_w16384", 100,
                                           ("lognormal", 3000.0, 0.8, 200, 20000),
                                           16384, SEED_BASE + 3),
}


def draw_toa_counts(rng: np.random.Generator, n_pulsars: int, law: tuple) -> np.ndarray:
    kind = law[0]
    if kind == "fixed":
        return np.full(n_pulsars, int(law[1]), dtype=np.int64)
    if kind == "uniform":
        return rng.integers(law[1], law[2] + 1, size=n_pulsars).astype(np.int64)
    if kind == "lognormal":
        med, s, lo, hi = law[1:]
        n = np.exp(np.log(med) + s * rng.standard_normal(n_pulsars))
        return np.clip(np.rint(n), lo, hi).astype(np.int64)
    raise ValueError(f"unknown TOA-count law {law!r}")


def draw_prior(rng: np.random.Generator, n_pulsars: int, n: int, model: str = "rw",
               pulsar_term: bool = False) -> np.ndarray:
    """n parameter vectors drawn uniformly from the prior box, float64 [n, D]."""
    pr = noise_prior(model, pulsar_term)
    k = len(pr)
    gw = PRIOR_GW[:, 0] + (PRIOR_GW[:, 1] - PRIOR_GW[:, 0]) * rng.random((n, N_GW))
    nz = pr[:, 0] + (pr[:, 1] - pr[:, 0]) * rng.random((n, n_pulsars, k))
    return np.concatenate([gw, nz.reshape(n, k * n_pulsars)], axis=1)


def isotropic_positions(rng: np.random.Generator, n: int) -> np.ndarray:
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sth = np.sqrt(1.0 - cth ** 2)
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def make_array(n_toa: np.ndarray, seed: int, with_signal: bool = True,
               t_obs: float = T_OBS, equad: float = 0.0, model: str = "rw",
               pulsar_term: bool = False) -> ArrayData:
    """Draw TOAs, errors, positions, a true parameter vector and residuals."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_toa = np.asarray(n_toa, dtype=np.int64)
    P = len(n_toa)
    theta = draw_prior(rng, P, 1, model)[0]
    k = 3 if model == "ou" else 2
    if not with_signal:
        theta[6] = -30.0   # negligible strain
    pos = isotropic_positions(rng, P)
    off = np.zeros(P + 1, dtype=np.int64)
    off[1:] = np.cumsum(n_toa)
    t = np.empty(off[-1]); r = np.empty(off[-1]); sig = np.full(off[-1], SIGMA_TOA)
    f_gw = 10.0 ** theta[0]
    amp0 = 10.0 ** theta[6] / (2.0 * np.pi * f_gw)
    for p in range(P):
        a, b = off[p], off[p + 1]
        n = b - a
        tp = np.sort(rng.uniform(0.0, t_obs, n))
        if n == 0:
            continue
        log10_sig, efac = theta[7 + k * p], theta[7 + k * p + k - 1]
        sp = 10.0 ** log10_sig
        dt = np.diff(tp, prepend=tp[0])
        if model == "ou":
            # Ornstein-Uhlenbeck fractional frequency, exact AR(1) steps
            gam = 10.0 ** theta[7 + k * p + 1]
            z = rng.standard_normal(n)
            y = np.empty(n)
            y[0] = np.sqrt(P0_DEFAULT[2]) * rng.standard_normal()
            for i in range(1, n):
                decay = np.exp(-gam * dt[i])
                y[i] = decay * y[i - 1] + sp * np.sqrt(-np.expm1(-2 * gam * dt[i]) / (2 * gam)) * z[i]
        else:
            # integrated random walk of the fractional frequency y
            y = np.sqrt(P0_DEFAULT[2]) * rng.standard_normal() + np.cumsum(sp * np.sqrt(dt) * rng.standard_normal(n))
        y_prev = np.concatenate([[y[0]], y[:-1]])
        rho = np.sqrt(P0_DEFAULT[0]) * rng.standard_normal() + np.cumsum(0.5 * dt * (y + y_prev))
        white = efac * sig[a:b] * rng.standard_normal(n)
        sinus = 0.0
        if with_signal:
            amp = amp0 * rng.uniform(0.3, 2.0)
            sinus = amp * np.sin(2.0 * np.pi * f_gw * tp + rng.uniform(0, 2 * np.pi))
        t[a:b] = tp; r[a:b] = rho + white + sinus
    # array epoch: earliest TOA of the whole array is t = 0
    t -= t.min()
    if pulsar_term:
        # distances drawn after everything else, so the residuals do not
        # depend on the flag
        d = PRIOR_DIST[0, 0] + (PRIOR_DIST[0, 1] - PRIOR_DIST[0, 0]) * rng.random(P)
        blocks = theta[N_GW:].reshape(P, k)
        theta = np.concatenate([theta[:N_GW], np.concatenate([blocks, d[:, None]], axis=1).ravel()])
    return ArrayData(off=off, t=t, r=r, sigma=sig, pos=pos,
                     equad=np.full(P, equad), p0=np.tile(np.array(P0_DEFAULT), (P, 1)),
                     theta_true=theta, model=model, pulsar_term=pulsar_term)


def make_workload_array(name: str, model: str = "rw", pulsar_term: bool = False) -> ArrayData:
    w = WORKLOADS[name]
    rng = np.random.Generator(np.random.PCG64(w.seed))
    n_toa = draw_toa_counts(rng, w.n_pulsars, w.toa_law)
    return make_array(n_toa, w.seed + 1000, with_signal=w.with_signal, model=model,
                      pulsar_term=pulsar_term)


def make_theta_batch(data: ArrayData, batch: int, seed: int, kind: str = "posterior") -> np.ndarray:
    """Parameter vectors float64 [batch, D].

    kind="posterior": the true vector plus a small Gaussian perturbation (states a
    sampler visits); kind="prior": independent prior draws.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    P = data.n_pulsars
    k = data.n_per_pulsar
    if kind == "prior":
        return draw_prior(rng, P, batch, data.model, data.pulsar_term)
    width = np.concatenate([
        np.array([1e-4, 1e-2, 1e-2, 1e-2, 1e-2, 1e-2, 1e-2]),
        np.tile(np.full(k, 1e-2), P)])
    th = data.theta_true[None, :] + width[None, :] * rng.standard_normal((batch, data.dim))
    # keep the bounded coordinates inside their domain
    th[:, 3] = np.clip(th[:, 3], -1.0, 1.0)
    th[:, 4] = np.clip(th[:, 4], -0.999, 0.999)
    th[:, 7 + data.efac_slot::k] = np.abs(th[:, 7 + data.efac_slot::k])
    if data.pulsar_term:
        th[:, 7 + k - 1::k] = np.abs(th[:, 7 + k - 1::k])
    return th
