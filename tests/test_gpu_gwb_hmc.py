"""End to end: batched HMC on the joint GW-background posterior, with the GPU
likelihood and its adjoint gradient at every leapfrog step, recovers the
parameters of data drawn from the model itself (the paper's workflow, on a
small synthetic array with a known injected background)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import dense
from paper_2510_11077_gb300 import inputs, sampler

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_hmc_recovers_an_injected_background():
    from paper_2510_11077_gb300 import argus, gwb_inference
    argus.load()
    P = 4
    data = inputs.make_array(np.full(P, 80), seed=601, equad=0.0)
    truth = np.concatenate([[-18.3, -8.2],
                            np.ravel([[-19.8, -8.8, 1.05], [-20.2, -8.1, 0.95],
                                      [-19.6, -9.2, 1.0], [-20.4, -7.9, 1.1]])])
    # residuals drawn from the model: N(0, C(truth)), C the dense covariance
    C = dense.gwb_covariance(data, truth)
    L = np.linalg.cholesky(C)
    data.r = L @ np.random.default_rng(7).standard_normal(len(data.r))
    target = gwb_inference.GwbTarget(data)
    out = gwb_inference.run_hmc(target, n_chains=256, n_warm=200, n_samp=150, n_steps=8, seed=3)
    s = out["samples"]                                   # [chains, draws, D]
    assert np.all(np.isfinite(s))
    assert 0.5 < out["accept"] < 0.99, out["accept"]
    flat = s.reshape(-1, s.shape[2])
    mean, sd = flat.mean(axis=0), flat.std(axis=0)
    # the injected amplitude and the white-noise levels are measured
    for j in (0, 4, 7, 10, 13):
        assert abs(mean[j] - truth[j]) < 4.0 * sd[j], (j, mean[j], sd[j], truth[j])
    assert sd[0] < 0.25 * (gwb_inference.PRIOR_GWB[0, 1] - gwb_inference.PRIOR_GWB[0, 0])
    # chains agree: effective sample size of the amplitude
    assert sampler.ess(s[:, :, [0]])[0] > 200
