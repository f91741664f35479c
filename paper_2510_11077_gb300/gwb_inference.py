"""Gradient-based inference with the joint likelihood of a Hellings-Downs
correlated GW background (argus_gwb.h): the paper's workflow, in which a
gradient-based sampler (the paper uses NUTS) calls the likelihood and its
gradient at every step, here as batched HMC over many chains, with every
call one GPU evaluation of the joint filter and its adjoint.

The prior is uniform on a box for every parameter; chains move in
unconstrained coordinates z, theta = lo + (hi - lo) sigmoid(z), with the
log-Jacobian added to the target (as the continuous-wave sampler does).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import argus, sampler
from .da_experiment import warmup

# prior box of the GW background and of each pulsar's own parameters
PRIOR_GWB = np.array([[-20.0, -17.0],    # log10 h_a [s^-1/2]
                      [-9.5, -7.0]])     # log10 gamma_a [1/s]
PRIOR_PULSAR = np.array([[-21.0, -19.0],     # log10 sigma_p
                         [-10.0, -7.0],      # log10 gamma_p
                         [0.8, 1.2]])        # EFAC


def prior_box(n_pulsars: int):
    lo = np.concatenate([PRIOR_GWB[:, 0], np.tile(PRIOR_PULSAR[:, 0], n_pulsars)])
    hi = np.concatenate([PRIOR_GWB[:, 1], np.tile(PRIOR_PULSAR[:, 1], n_pulsars)])
    return lo, hi


class GwbTarget:
    """log p(z) = joint loglik(theta(z)) + sum log(dtheta/dz), and its gradient."""

    def __init__(self, data, device: int = 0):
        self.arr = argus.GwbArray(data, device=device)
        lo, hi = prior_box(data.n_pulsars)
        dev = torch.device("cuda", device)
        self.lo = torch.tensor(lo, dtype=torch.float64, device=dev)
        self.hi = torch.tensor(hi, dtype=torch.float64, device=dev)
        self.calls = 0

    def to_theta(self, z):
        return self.lo + (self.hi - self.lo) * torch.sigmoid(z)

    def to_z(self, theta):
        u = ((theta - self.lo) / (self.hi - self.lo)).clamp(1e-12, 1 - 1e-12)
        return torch.log(u) - torch.log1p(-u)

    def logp_grad(self, z):
        sg = torch.sigmoid(z)
        dtdz = (self.hi - self.lo) * sg * (1 - sg)
        ll, g = argus.argus_gwb_loglik_grad(self.arr, self.to_theta(z).contiguous())
        self.calls += z.shape[0]
        lp = ll + torch.log(dtdz).sum(dim=1)
        lp = torch.where(torch.isfinite(lp), lp, torch.full_like(lp, -math.inf))
        return lp, g * dtdz + (1 - 2 * sg)


def run_hmc(target: GwbTarget, n_chains: int, n_warm: int, n_samp: int, n_steps: int, seed: int,
            log=None):
    """Warm-up (dual-averaged step size, diagonal mass) then n_samp HMC
    iterations per chain.  Returns dict(samples [C, n_samp, D] in theta,
    accept, eps, seconds, gradient_evals)."""
    dev = target.lo.device
    D = target.lo.shape[0]
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    z0 = 0.5 * torch.randn((n_chains, D), generator=gen, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st, eps, inv_mass, _ = warmup(target, z0, n_warm, n_steps, gen, log=log)
    eps_t = torch.full((n_chains, 1), eps, dtype=torch.float64, device=dev)
    draws, acc = [], []
    for _ in range(n_samp):
        st, a = sampler.hmc_step(st, target.logp_grad, eps_t, n_steps, inv_mass, gen)
        draws.append(target.to_theta(st.x))
        acc.append(a.mean())
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    samples = torch.stack(draws, dim=1).cpu().numpy()
    return {"samples": samples, "accept": float(torch.stack(acc).mean()), "eps": eps,
            "seconds": secs, "gradient_evals": target.calls}
