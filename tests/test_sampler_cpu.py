"""Sampler pins on CPU: HMC and delayed-acceptance HMC against Gaussian
targets with known moments (the second with a deliberately wrong
approximation in stage 1), and the ESS estimator against AR(1) chains with a
closed-form integrated autocorrelation time."""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2510_11077_gb300 import sampler  # noqa: E402

D = 4
MEAN = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64)
L = torch.tensor([[1.0, 0, 0, 0], [0.6, 0.8, 0, 0], [-0.3, 0.2, 0.5, 0], [0.1, 0.0, 0.4, 2.0]],
                 dtype=torch.float64)
COV = L @ L.T
PREC = torch.linalg.inv(COV)


def gauss(x):
    d = x - MEAN
    lp = -0.5 * torch.einsum("ci,ij,cj->c", d, PREC, d)
    return lp, -d @ PREC


def wrong_gauss(x):
    """An approximation with a shifted mean, wrong scale and no correlation."""
    d = x - MEAN - 0.3
    s = torch.tensor([1.5, 0.7, 1.0, 1.3], dtype=torch.float64)
    return -0.5 * torch.sum((d / s) ** 2, dim=1), -d / s ** 2


def _run(kind, iters=400, chains=512, seed=0, dense=False):
    gen = torch.Generator().manual_seed(seed)
    x = MEAN + torch.randn((chains, D), generator=gen, dtype=torch.float64)
    inv_mass = sampler.DenseMass(COV.clone()) if dense else torch.diag(COV)[None, :].clone()
    eps = torch.full((chains, 1), 0.35, dtype=torch.float64)
    if kind == "hmc":
        st = sampler.ChainState(x, *gauss(x))
    else:
        lps, gs = wrong_gauss(x)
        st = sampler.DAState(x, lps, gs, gauss(x)[0])
    draws, accs = [], []
    for it in range(iters):
        if kind == "hmc":
            st, a = sampler.hmc_step(st, gauss, eps, 8, inv_mass, gen)
        else:
            st, _, a, _ = sampler.da_hmc_step(st, wrong_gauss, lambda z: gauss(z)[0], eps, 8, inv_mass, gen)
        accs.append(float(a.mean()))
        if it >= 100:
            draws.append(st.x.clone())
    return torch.stack(draws, dim=1).numpy(), np.mean(accs)


@pytest.mark.parametrize("kind,dense", [("hmc", False), ("da", False), ("hmc", True), ("da", True)])
def test_samplers_recover_gaussian_moments(kind, dense):
    s, acc = _run(kind, dense=dense)
    C, T, _ = s.shape
    flat = s.reshape(-1, D)
    # antithetic mixing can push the estimate above the draw count; cap it there
    ess = np.minimum(sampler.ess(s), C * T)
    mcse = np.sqrt(np.diag(COV.numpy()) / ess)
    assert np.all(np.abs(flat.mean(0) - MEAN.numpy()) < 5 * mcse), (flat.mean(0), mcse)
    # each covariance entry is the mean of a product series; its Monte Carlo
    # error uses that series' own ESS (antithetic moves help means, not variances)
    S = COV.numpy()
    xc = s - s.reshape(-1, D).mean(0)
    for i in range(D):
        for j in range(i, D):
            prod = xc[:, :, i] * xc[:, :, j]
            e = min(sampler.ess(prod[:, :, None])[0], C * T)
            se = prod.std() / np.sqrt(e)
            assert abs(prod.mean() - S[i, j]) < 5 * se + 1e-3 * abs(S[i, i] * S[j, j]) ** 0.5, (i, j)
    assert acc > 0.2


def test_delayed_acceptance_saves_exact_calls_when_the_approximation_is_bad():
    gen = torch.Generator().manual_seed(3)
    x = MEAN + torch.randn((1000, D), generator=gen, dtype=torch.float64)
    st = sampler.DAState(x, *wrong_gauss(x), gauss(x)[0])
    inv_mass = torch.diag(COV)[None, :].clone()
    eps = torch.full((1000, 1), 0.35, dtype=torch.float64)
    n_exact = 0
    for _ in range(30):
        st, a1, a, n = sampler.da_hmc_step(st, wrong_gauss, lambda z: gauss(z)[0], eps, 8, inv_mass, gen)
        n_exact += n
    assert n_exact < 30 * 1000          # stage 1 screens some proposals out


def test_ess_matches_ar1_closed_form():
    rng = np.random.default_rng(0)
    C, T = 256, 2000
    for rho in (0.0, 0.5, 0.9):
        e = rng.standard_normal((C, T))
        x = np.empty((C, T))
        x[:, 0] = e[:, 0] / math.sqrt(1 - rho ** 2) if rho else e[:, 0]
        for t in range(1, T):
            x[:, t] = rho * x[:, t - 1] + e[:, t]
        est = sampler.ess(x[:, :, None])[0]
        exact = C * T * (1 - rho) / (1 + rho)
        assert abs(est / exact - 1) < 0.1, (rho, est, exact)


def test_dual_averaging_reaches_target_acceptance():
    gen = torch.Generator().manual_seed(5)
    x = MEAN + torch.randn((256, D), generator=gen, dtype=torch.float64)
    st = sampler.ChainState(x, *gauss(x))
    inv_mass = torch.ones((1, D), dtype=torch.float64)
    da = sampler.DualAveraging(0.05, target=0.8)
    eps = 0.05
    for _ in range(300):
        st, a = sampler.hmc_step(st, gauss, torch.full((256, 1), eps, dtype=torch.float64), 6,
                                 inv_mass, gen)
        eps = da.update(float(a.mean()))
    eps = da.final()
    accs = []
    for _ in range(100):
        st, a = sampler.hmc_step(st, gauss, torch.full((256, 1), eps, dtype=torch.float64), 6,
                                 inv_mass, gen)
        accs.append(float(a.mean()))
    assert abs(np.mean(accs) - 0.8) < 0.08


def test_dense_mass_kinetic_energy_and_momentum_law():
    gen = torch.Generator().manual_seed(9)
    m = sampler.DenseMass(COV.clone())
    p = m.sample((200000, D), gen, torch.float64, "cpu")
    # p ~ N(0, COV^-1): E[p p^T] = PREC, and E[kinetic] = D / 2
    assert torch.allclose(p.T @ p / p.shape[0], PREC, atol=0.03 * PREC.abs().max())
    assert abs(float(m.kinetic(p).mean()) - D / 2) < 0.02 * D
