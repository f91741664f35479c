"""Batched Hamiltonian Monte Carlo and delayed-acceptance HMC.

The paper's sampler integration calls the likelihood and its gradient at
every step of a gradient-based sampler (HMC / NUTS).  Here many chains move
in lock-step so that every likelihood call is one batched GPU evaluation.

* `hmc_step`: one HMC transition per chain (leapfrog with L steps, momentum
  refresh, Metropolis accept with the exact Hamiltonian).
* `da_hmc_step`: delayed acceptance (Christen & Fox 2005) with a cheap
  approximate target: the leapfrog trajectory is integrated with the
  approximation's gradient; stage 1 accepts with the approximation's
  Hamiltonian, and only stage-1 survivors are evaluated exactly; stage 2
  accepts with min(1, exp(dH_exact - dH_approx)).  Leapfrog with any smooth
  vector field followed by a momentum flip is a volume-preserving
  involution, so the two-stage rule leaves the exact target invariant; the
  approximation only changes the acceptance rate.
* `dual_averaging`: step-size adaptation to a target acceptance rate
  (Hoffman & Gelman 2014).
* `ess`: multi-chain effective sample size with Geyer's initial monotone
  sequence (as in Stan / Vehtari et al. 2021, without rank normalization).

Targets are callables `logp(x) -> (lp [C], grad [C, D])` on torch tensors;
`-inf` log-density means outside the support (always rejected).
"""
from __future__ import annotations

import math

import numpy as np
import torch


class DenseMass:
    """Kinetic energy p^T S p / 2 with S = inverse mass (e.g. a posterior
    covariance); momenta p ~ N(0, S^-1) drawn as z L^-1 with S = L L^T."""

    def __init__(self, S):
        self.S = S
        self.Linv = torch.linalg.inv(torch.linalg.cholesky(S))

    def sample(self, shape, gen, dtype, device):
        z = torch.randn(shape, generator=gen, dtype=dtype, device=device)
        return z @ self.Linv

    def kinetic(self, p):
        return 0.5 * torch.sum((p @ self.S) * p, dim=1)

    def velocity(self, p):
        return p @ self.S


def _sample_p(x, inv_mass, gen):
    if isinstance(inv_mass, DenseMass):
        return inv_mass.sample(x.shape, gen, x.dtype, x.device)
    return torch.randn(x.shape, generator=gen, dtype=x.dtype, device=x.device) / torch.sqrt(inv_mass)


def _kinetic(p, inv_mass):
    if isinstance(inv_mass, DenseMass):
        return inv_mass.kinetic(p)
    return 0.5 * torch.sum(p * p * inv_mass, dim=1)


def _velocity(p, inv_mass):
    return inv_mass.velocity(p) if isinstance(inv_mass, DenseMass) else inv_mass * p


def leapfrog(x, p, lp, g, logp_grad, eps, n_steps, inv_mass):
    """L leapfrog steps from (x, p) with cached (lp, g) at x; eps [C, 1];
    inv_mass a [1, D] diagonal or a DenseMass."""
    p = p + 0.5 * eps * g
    for i in range(n_steps):
        x = x + eps * _velocity(p, inv_mass)
        lp, g = logp_grad(x)
        if i < n_steps - 1:
            p = p + eps * g
    p = p + 0.5 * eps * g
    return x, p, lp, g


def _finite(v):
    return torch.where(torch.isfinite(v), v, torch.full_like(v, -math.inf))


class ChainState:
    """Positions and the cached log-density / gradient of each chain."""

    def __init__(self, x, lp, g):
        self.x, self.lp, self.g = x, lp, g


def hmc_step(state, logp_grad, eps, n_steps, inv_mass, gen):
    """One exact HMC transition for every chain.  Returns (state, accept_prob)."""
    x, lp, g = state.x, state.lp, state.g
    C = x.shape[0]
    p = _sample_p(x, inv_mass, gen)
    h0 = -lp + _kinetic(p, inv_mass)
    x1, p1, lp1, g1 = leapfrog(x, p, lp, g, logp_grad, eps, n_steps, inv_mass)
    lp1 = _finite(lp1)
    h1 = -lp1 + _kinetic(p1, inv_mass)
    a = torch.exp(torch.clamp(h0 - h1, max=0.0))
    a = torch.where(torch.isfinite(h1), a, torch.zeros_like(a))
    u = torch.rand(C, generator=gen, dtype=x.dtype, device=x.device)
    acc = u < a
    m = acc[:, None]
    return ChainState(torch.where(m, x1, x), torch.where(acc, lp1, lp), torch.where(m, g1, g)), a


class DAState:
    """Chain positions with the approximate (lp, g) and exact lp at each."""

    def __init__(self, x, lp_s, g_s, lp_e):
        self.x, self.lp_s, self.g_s, self.lp_e = x, lp_s, g_s, lp_e


class GraphedLeapfrog:
    """`leapfrog` for a fixed batch shape, captured once in a CUDA graph and
    replayed (the trajectory's kernels launch without per-step host work).
    The captured target must run only stream-ordered GPU work."""

    def __init__(self, logp_grad, n_steps, inv_mass, shape, dtype, device, warmup=2):
        C, D = shape
        self.inp = [torch.zeros((C, D), dtype=dtype, device=device),      # x
                    torch.zeros((C, D), dtype=dtype, device=device),      # p
                    torch.zeros(C, dtype=dtype, device=device),           # lp
                    torch.zeros((C, D), dtype=dtype, device=device),      # g
                    torch.zeros((C, 1), dtype=dtype, device=device)]      # eps
        self.n_steps, self.inv_mass, self.logp_grad = n_steps, inv_mass, logp_grad
        side = torch.cuda.Stream(device)
        side.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                leapfrog(*self.inp[:4], logp_grad, self.inp[4], n_steps, inv_mass)
        torch.cuda.current_stream(device).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self.out = leapfrog(*self.inp[:4], logp_grad, self.inp[4], n_steps, inv_mass)

    def __call__(self, x, p, lp, g, logp_grad, eps, n_steps, inv_mass):
        assert logp_grad == self.logp_grad and n_steps == self.n_steps
        for dst, src in zip(self.inp, (x, p, lp, g, eps)):
            dst.copy_(src)
        self.graph.replay()
        return tuple(t.clone() for t in self.out)


def da_hmc_step(state, approx_logp_grad, exact_logp, eps, n_steps, inv_mass, gen,
                leapfrog_fn=None):
    """One delayed-acceptance HMC transition.

    approx_logp_grad(x) -> (lp, g): the cheap approximation (drives the
    trajectory and stage 1); exact_logp(x) -> lp: the exact log-density, called
    only on stage-1 survivors.  Returns (state, stage-1 prob, overall accept,
    number of exact evaluations).
    """
    x = state.x
    C = x.shape[0]
    p = _sample_p(x, inv_mass, gen)
    k0 = _kinetic(p, inv_mass)
    lf = leapfrog_fn or leapfrog
    x1, p1, lps1, gs1 = lf(x, p, state.lp_s, state.g_s, approx_logp_grad, eps, n_steps, inv_mass)
    lps1 = _finite(lps1)
    k1 = _kinetic(p1, inv_mass)
    dhs = (-state.lp_s + k0) - (-lps1 + k1)          # H_s(x, p) - H_s(x', p')
    a1 = torch.exp(torch.clamp(dhs, max=0.0))
    a1 = torch.where(torch.isfinite(dhs), a1, torch.zeros_like(a1))
    u1 = torch.rand(C, generator=gen, dtype=x.dtype, device=x.device)
    pass1 = u1 < a1
    idx = torch.nonzero(pass1).flatten()
    lpe1 = torch.full_like(state.lp_e, -math.inf)
    if idx.numel() > 0:
        lpe1[idx] = _finite(exact_logp(x1[idx].contiguous()))
    dhe = (-state.lp_e + k0) - (-lpe1 + k1)
    log_a2 = torch.where(pass1, dhe - dhs, torch.full_like(dhe, -math.inf))
    a2 = torch.nan_to_num(torch.exp(torch.clamp(log_a2, max=0.0)), nan=0.0)
    u2 = torch.rand(C, generator=gen, dtype=x.dtype, device=x.device)
    acc = pass1 & (u2 < a2)
    m = acc[:, None]
    new = DAState(torch.where(m, x1, x), torch.where(acc, lps1, state.lp_s),
                  torch.where(m, gs1, state.g_s), torch.where(acc, lpe1, state.lp_e))
    return new, a1, a1 * a2, int(idx.numel())


class DualAveraging:
    """Step-size adaptation towards a target mean acceptance (Hoffman & Gelman 2014)."""

    def __init__(self, eps0, target=0.8, gamma=0.05, t0=10.0, kappa=0.75):
        self.mu = math.log(10.0 * eps0)
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.hbar = 0.0
        self.logeps = math.log(eps0)
        self.logeps_bar = 0.0
        self.m = 0

    def update(self, accept_mean):
        self.m += 1
        w = 1.0 / (self.m + self.t0)
        self.hbar = (1 - w) * self.hbar + w * (self.target - accept_mean)
        self.logeps = self.mu - math.sqrt(self.m) / self.gamma * self.hbar
        eta = self.m ** (-self.kappa)
        self.logeps_bar = eta * self.logeps + (1 - eta) * self.logeps_bar
        return math.exp(self.logeps)

    def final(self):
        return math.exp(self.logeps_bar)


def ess(samples):
    """Multi-chain effective sample size per dimension.

    samples: array [chains, draws, dims].  Autocovariances by FFT within each
    chain, combined with the between-chain variance, summed over Geyer's
    initial positive and monotone sequence of paired autocorrelations.
    """
    x = np.asarray(samples, dtype=np.float64)
    C, T, D = x.shape
    if T < 4:
        raise ValueError("need at least 4 draws per chain")
    xc = x - x.mean(axis=1, keepdims=True)
    n = 1 << (2 * T - 1).bit_length()
    f = np.fft.rfft(xc, n=n, axis=1)
    acov = np.fft.irfft(f * np.conj(f), n=n, axis=1)[:, :T, :] / T      # [C, T, D]
    chain_var = acov[:, 0, :] * T / (T - 1)
    W = chain_var.mean(axis=0)
    Bt = x.mean(axis=1).var(axis=0, ddof=1) if C > 1 else np.zeros(D)
    var_plus = (T - 1) / T * W + Bt
    rho = 1.0 - (W[None, :] - acov.mean(axis=0)) / var_plus[None, :]     # [T, D]
    rho[0] = 1.0
    out = np.empty(D)
    for d in range(D):
        r = rho[:, d]
        tau = -1.0
        prev = math.inf
        for k in range(0, T - 1, 2):
            pk = r[k] + r[k + 1]
            if pk < 0:
                break
            pk = min(pk, prev)
            tau += 2.0 * pk
            prev = pk
        out[d] = C * T / max(tau, 1e-12)
    return out
