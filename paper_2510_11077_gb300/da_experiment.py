"""Surrogate-accelerated delayed-acceptance HMC on a 20-pulsar array.

1. Exact HMC warm-up (all chains in lock-step) with dual-averaging step size
   and a diagonal mass matrix from the warm-up draws.
2. Training set: points drawn around the warm-up posterior (Gaussian with
   `spread` x its covariance), each evaluated by the exact FP64 filter
   (loglik + gradient).
   Sampling, training and the surrogate all work in unconstrained
   coordinates z (theta = lo + (hi - lo) sigmoid(z) for the uniform prior box).
3. Surrogate training on the GPU (BF16 tensor-core MLP, Adam).
4. From the same warmed-up state: plain exact HMC and delayed-acceptance HMC
   (surrogate trajectory and stage 1, exact filter as stage 2), both with the
   same step size, mass matrix and trajectory length.
5. ESS/s (minimum over parameters) of both, with and without the surrogate's
   data-generation and training time, and a check that the two posteriors
   agree (means within Monte Carlo error).

The network sees FP32 inputs; to keep their precision it is fed parameter
offsets from a fixed FP64 centre and log-likelihood offsets from a fixed FP64
reference value.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import argus, inputs, sampler
from .surrogate import Surrogate

N_GW = inputs.N_GW


def prior_box(P):
    lo = np.concatenate([inputs.PRIOR_GW[:, 0], np.tile(inputs.PRIOR_NOISE[:, 0], P)])
    hi = np.concatenate([inputs.PRIOR_GW[:, 1], np.tile(inputs.PRIOR_NOISE[:, 1], P)])
    return lo, hi


class ExactTarget:
    """Exact FP64 filter posterior in unconstrained coordinates z.

    Every parameter has a uniform prior on a box [lo, hi]; sampling runs in
    z with theta = lo + (hi - lo) sigmoid(z), so the target is
    log p(z) = ll(theta(z)) + sum log(dtheta/dz) and no trajectory meets a
    wall.
    """

    def __init__(self, data, device):
        self.arr = argus.Array(data, device=device)      # loglik + grad, graph replay
        self.arr.set_plan(tape_cache=1, walkers_per_cta=32, ctas_per_sm=12)
        self.arr_ll = argus.Array(data, device=device)   # loglik of varying batch sizes
        # small tiles balance the stage-1 survivors' uneven batches over the SMs
        self.arr_ll.set_plan(use_graph=0, walkers_per_cta=32, ctas_per_sm=12)
        lo, hi = prior_box(data.n_pulsars)
        self.lo = torch.tensor(lo, dtype=torch.float64, device=device)
        self.hi = torch.tensor(hi, dtype=torch.float64, device=device)
        self.calls_grad = 0
        self.calls_ll = 0
        self._bufs = {}

    def to_theta(self, z):
        return self.lo + (self.hi - self.lo) * torch.sigmoid(z)

    def to_z(self, theta):
        u = ((theta - self.lo) / (self.hi - self.lo)).clamp(1e-12, 1 - 1e-12)
        return torch.log(u) - torch.log1p(-u)

    def _jac(self, z):
        sg = torch.sigmoid(z)
        dtdz = (self.hi - self.lo) * sg * (1 - sg)
        return torch.log(dtdz).sum(dim=1), dtdz, 1 - 2 * sg

    def loglik_grad(self, theta):
        """Exact loglik + gradient in theta, through fixed buffers (one captured
        graph per batch size is replayed instead of re-captured)."""
        B, D = theta.shape
        if B not in self._bufs:
            dev = theta.device
            self._bufs[B] = (torch.empty((B, D), dtype=torch.float64, device=dev),
                             torch.empty(B, dtype=torch.float64, device=dev),
                             torch.empty((B, D), dtype=torch.float64, device=dev))
        th, ll, g = self._bufs[B]
        th.copy_(theta)
        argus.argus_loglik_grad(self.arr, th, ll, g)
        return ll.clone(), g.clone()

    def logp_grad(self, z):
        ll, g = self.loglik_grad(self.to_theta(z))
        self.calls_grad += z.shape[0]
        lj, dtdz, glj = self._jac(z)
        lp = ll + lj
        lp = torch.where(torch.isfinite(lp), lp, torch.full_like(lp, -math.inf))
        return lp, g * dtdz + glj

    def logp(self, z):
        ll = argus.argus_loglik(self.arr_ll, self.to_theta(z).contiguous())
        self.calls_ll += z.shape[0]
        lp = ll + self._jac(z)[0]
        return torch.where(torch.isfinite(lp), lp, torch.full_like(lp, -math.inf))


class SurrogateTarget:
    """The same log posterior in z approximated by the trained network (fed the
    offset from a fixed FP64 centre, and returning the offset from ll_ref)."""

    def __init__(self, net, exact, centre, ll_ref):
        self.net, self.exact = net, exact
        self.centre = centre
        self.ll_ref = ll_ref

    def logp_grad(self, z):
        # float(z - centre) in, value + ll_ref and its gradient out, all in the
        # fused kernel (the same rounding as converting around argus_surrogate_eval)
        return self.net.eval_z(z, self.centre, self.ll_ref)


def _sync():
    torch.cuda.synchronize()


def model_array(seed, log10_h0=-13.7, device=0):
    """The 20-pulsar workload's TOAs and noise, plus the model's own
    continuous-wave residual at a detectable strain, so that the posterior is
    centred on known parameters.  Returns (data, theta_true)."""
    w = inputs.WORKLOADS["psr20_toa500-2000_w4096"]
    rng = np.random.Generator(np.random.PCG64(w.seed))
    n_toa = inputs.draw_toa_counts(rng, w.n_pulsars, w.toa_law)
    data = inputs.make_array(n_toa, seed, with_signal=False)
    theta = data.theta_true.copy()
    theta[6] = log10_h0
    arr = argus.Array(data, device=device)
    data.r = data.r + argus.argus_cw_signal(arr, theta[:N_GW], int(data.off[-1]))
    arr.close()
    data.theta_true = theta
    return data, theta


def warmup(target, x0, n_iter, n_steps, gen, log=None):
    """Exact HMC warm-up: dual averaging of the step size; diagonal mass from the
    second half of the draws (re-estimated once at 60%)."""
    C, D = x0.shape
    inv_mass = x0.var(dim=0, keepdim=True).clamp_min(1e-30)   # initial scales from the starts
    st = sampler.ChainState(x0, *target.logp_grad(x0))
    da = sampler.DualAveraging(0.05, target=0.8)
    eps = 0.05
    keep = []
    tail = []
    for it in range(n_iter):
        st, a = sampler.hmc_step(st, target.logp_grad, torch.full((C, 1), eps, dtype=torch.float64,
                                                                  device=x0.device),
                                 n_steps, inv_mass, gen)
        eps = da.update(float(a.mean()))
        if it >= n_iter // 3:
            keep.append(st.x)
        if it >= int(0.75 * n_iter):
            tail.append(st.x)
        if it == int(0.6 * n_iter) and keep:
            xs = torch.stack(keep)
            inv_mass = xs.reshape(-1, D).var(dim=0, keepdim=True).clamp_min(1e-30)
            keep = []
            da = sampler.DualAveraging(eps, target=0.8)
        if log and it % 25 == 0:
            log(f"warmup {it}: eps {eps:.3g} acc {float(a.mean()):.3f}")
    return st, da.final(), inv_mass, torch.cat(tail)


def make_training_set(target, centre, chol, n, batch, gen):
    """n exact (log posterior, gradient) evaluations at centre + chol N(0, I) in z."""
    D = centre.shape[0]
    xs, lls, gs = [], [], []
    done = 0
    while done < n:
        b = min(batch, n - done)
        z = torch.randn((b, D), generator=gen, dtype=torch.float64, device=centre.device)
        x = centre[None, :] + z @ chol.T
        ll, g = target.logp_grad(x)
        ok = torch.isfinite(ll)
        xs.append(x[ok]); lls.append(ll[ok]); gs.append(g[ok])
        done += b
    return torch.cat(xs), torch.cat(lls), torch.cat(gs)


def train(net, x, ll, g, centre, ll_ref, epochs, batch, lr, gen, log=None):
    n = x.shape[0]
    u = (x - centre).float()
    llc = (ll - ll_ref).float()
    gf = g.float()
    losses = []
    steps = epochs * (n // batch)
    for name, a in (("inputs", u), ("loglik", llc), ("grad", gf)):
        if not bool(torch.isfinite(a).all()):
            raise FloatingPointError(f"non-finite training {name}")
    k = 0
    loss_buf = torch.empty(1, dtype=torch.float32, device=x.device)
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=x.device)
        # the epoch's shuffled copy, so that each minibatch is a contiguous slice
        up, lp, gp = u[perm], llc[perm], gf[perm]
        for i in range(n // batch):
            sl = slice(i * batch, (i + 1) * batch)
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps))    # cosine decay
            loss = net.train_step(up[sl], lp[sl], gp[sl], lr_k, loss_out=loss_buf)
            k += 1
        losses.append(float(loss.item()))
        if not math.isfinite(losses[-1]):
            raise FloatingPointError(f"training loss became {losses[-1]} in epoch {ep}")
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4g}")
    net.check()
    return losses


def holdout_error(net, target, centre, ll_ref, x, ll, g):
    st = SurrogateTarget(net, target, centre, ll_ref)
    lp, gp = st.logp_grad(x)
    err = (lp - ll).abs()
    gerr = (gp - g).norm(dim=1) / g.norm(dim=1).clamp_min(1e-30)
    return float(err.median()), float(err.quantile(0.9)), float(gerr.median())


def run(n_chains=4096, n_train=1_000_000, warmup_iter=200, sample_iter=100, da_iter=None,
        n_steps=16,
        spread=1.0, epochs=40, batch=4096, lr=1e-3, value_weight=10.0, seed=20251017, device=0,
        retune_iter=40, grad_mode=1, graph_leapfrog=True, log=None):
    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    gen = torch.Generator(device=dev).manual_seed(seed)
    data, theta_true = model_array(seed, device=device)
    target = ExactTarget(data, device)
    D = data.dim
    assert D == 47
    th0 = torch.from_numpy(inputs.make_theta_batch(data, n_chains, seed=seed)).to(dev)
    x0 = target.to_z(torch.maximum(torch.minimum(th0, target.hi), target.lo))
    t0 = time.perf_counter()
    st, eps, inv_mass, draws_w = warmup(target, x0, warmup_iter, n_steps, gen, log)
    _sync()
    t_warm = time.perf_counter() - t0
    # Gaussian approximation of the posterior from the last warm-up draws
    centre = draws_w.mean(dim=0)
    cov = torch.cov(draws_w.T) + torch.diag(1e-12 * torch.diag(torch.cov(draws_w.T)).clamp_min(1e-300))
    chol = torch.linalg.cholesky(cov)
    H = torch.linalg.inv(cov)
    ll_ref = float(st.lp.max())
    # dense mass from the same covariance; re-tune the step size under it
    mass = sampler.DenseMass(cov)
    da_eps = sampler.DualAveraging(eps, target=0.8)
    for it in range(retune_iter):
        st, a = sampler.hmc_step(st, target.logp_grad, torch.full((n_chains, 1), eps,
                                                                  dtype=torch.float64, device=dev),
                                 n_steps, mass, gen)
        eps = da_eps.update(float(a.mean()))
    if retune_iter:
        eps = da_eps.final()
    inv_mass = mass

    # training data from the exact filter
    t0 = time.perf_counter()
    xt, llt, gt = make_training_set(target, centre, spread * chol, n_train, 16384, gen)
    _sync()
    t_data = time.perf_counter() - t0
    n_hold = min(20000, xt.shape[0] // 10)
    xh, llh, gh = xt[:n_hold], llt[:n_hold], gt[:n_hold]
    xt, llt, gt = xt[n_hold:], llt[n_hold:], gt[n_hold:]
    net = Surrogate(device=device, max_rows=max(batch, n_chains), seed=seed)
    net.set_baseline(H.float().cpu().numpy())
    u = (xt - centre)
    resid = (llt - ll_ref) + 0.5 * torch.einsum("ni,ij,nj->n", u, H, u)   # target minus baseline
    net.set_normalizers(np.zeros(D, np.float32), u.std(dim=0).cpu().numpy().astype(np.float32),
                        float(resid.mean()), float(resid.std()), value_weight=value_weight,
                        grad_weight=1.0)
    t0 = time.perf_counter()
    losses = train(net, xt, llt, gt, centre, ll_ref, epochs, batch, lr, gen, log)
    _sync()
    t_train = time.perf_counter() - t0
    med, p90, gmed = holdout_error(net, target, centre, ll_ref, xh, llh, gh)

    eps_t = torch.full((n_chains, 1), eps, dtype=torch.float64, device=dev)
    # plain exact HMC
    st_h = sampler.ChainState(st.x.clone(), st.lp.clone(), st.g.clone())
    draws_h, acc_h = [], []
    _sync(); t0 = time.perf_counter()
    for _ in range(sample_iter):
        st_h, a = sampler.hmc_step(st_h, target.logp_grad, eps_t, n_steps, inv_mass, gen)
        draws_h.append(st_h.x)
        acc_h.append(a.mean())
    _sync(); t_hmc = time.perf_counter() - t0
    # delayed acceptance (grad_mode 1: trajectories follow the gradient of the
    # surrogate's own value output, so they conserve its energy)
    net.set_grad_mode(grad_mode)
    sur = SurrogateTarget(net, target, centre, ll_ref)
    lf = (sampler.GraphedLeapfrog(sur.logp_grad, n_steps, inv_mass, tuple(st.x.shape), st.x.dtype, dev)
          if graph_leapfrog else None)
    lps, gs = sur.logp_grad(st.x)
    st_d = sampler.DAState(st.x.clone(), lps, gs, st.lp.clone())
    draws_d, acc1_d, acc_d, n_exact = [], [], [], 0
    da_iter = da_iter or sample_iter
    _sync(); t0 = time.perf_counter()
    for _ in range(da_iter):
        st_d, a1, a, ne = sampler.da_hmc_step(st_d, sur.logp_grad, target.logp, eps_t, n_steps,
                                              inv_mass, gen, leapfrog_fn=lf)
        draws_d.append(st_d.x)
        acc1_d.append(a1.mean()); acc_d.append(a.mean())
        n_exact += ne
    _sync(); t_da = time.perf_counter() - t0

    dh = target.to_theta(torch.stack(draws_h, dim=1)).cpu().numpy()
    dd = target.to_theta(torch.stack(draws_d, dim=1)).cpu().numpy()
    ess_h = sampler.ess(dh)
    ess_d = sampler.ess(dd)
    # posterior agreement: difference of means in units of the combined MC error
    var = dh.reshape(-1, D).var(axis=0)
    se = np.sqrt(var / np.minimum(ess_h, dh.shape[0] * dh.shape[1]) +
                 dd.reshape(-1, D).var(axis=0) / np.minimum(ess_d, dd.shape[0] * dd.shape[1]))
    z = np.abs(dh.reshape(-1, D).mean(0) - dd.reshape(-1, D).mean(0)) / np.maximum(se, 1e-300)
    sd_ratio = np.sqrt(dd.reshape(-1, D).var(axis=0) / var)
    res = {
        "chains": n_chains, "dim": D, "leapfrog_steps": n_steps, "step_size": eps,
        "mass": "dense (warm-up covariance)",
        "surrogate_gradient": "back-propagated value output" if grad_mode == 1 else "gradient outputs",
        "da_leapfrog": "CUDA graph" if graph_leapfrog else "eager",
        "sample_iters": sample_iter, "da_iters": da_iter, "warmup_iters": warmup_iter,
        "warmup_s": t_warm,
        "train_rows": int(xt.shape[0]), "holdout_rows": int(n_hold), "epochs": epochs,
        "baseline": "Gaussian from the warm-up draws (network fits the residual)",
        "data_gen_s": t_data, "train_s": t_train, "final_loss": losses[-1],
        "holdout_abs_err_nats_median": med, "holdout_abs_err_nats_p90": p90,
        "holdout_grad_rel_err_median": gmed,
        "hmc": {"seconds": t_hmc, "accept": float(torch.stack(acc_h).mean()),
                "ess_min": float(ess_h.min()), "ess_median": float(np.median(ess_h)),
                "ess_per_s": float(ess_h.min() / t_hmc),
                "exact_grad_evals": sample_iter * n_steps * n_chains},
        "da_hmc": {"seconds": t_da, "accept_stage1": float(torch.stack(acc1_d).mean()),
                   "accept": float(torch.stack(acc_d).mean()),
                   "ess_min": float(ess_d.min()), "ess_median": float(np.median(ess_d)),
                   "ess_per_s": float(ess_d.min() / t_da),
                   "ess_per_s_incl_training": float(ess_d.min() / (t_da + t_data + t_train)),
                   "exact_ll_evals": n_exact,
                   "surrogate_evals": da_iter * n_steps * n_chains},
        "posterior_mean_z_max": float(z.max()),
        "posterior_sd_ratio_range": [float(sd_ratio.min()), float(sd_ratio.max())],
    }
    res["ess_per_s_gain"] = res["da_hmc"]["ess_per_s"] / max(res["hmc"]["ess_per_s"], 1e-300)
    res["ess_per_s_gain_incl_training"] = (res["da_hmc"]["ess_per_s_incl_training"] /
                                           max(res["hmc"]["ess_per_s"], 1e-300))
    net.close()
    return res
