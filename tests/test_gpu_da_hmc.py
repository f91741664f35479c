"""Delayed-acceptance HMC with the trained surrogate against plain exact HMC on
the 20-pulsar array (reduced sizes): the two posteriors agree within Monte
Carlo error, and the surrogate reaches useful accuracy."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_da_hmc_matches_exact_hmc_posterior():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_11077_gb300 import da_experiment
    res = da_experiment.run(n_chains=1024, n_train=300_000, warmup_iter=120, sample_iter=60,
                            da_iter=120, n_steps=12, epochs=30, batch=4096, log=print)
    print(res)
    assert res["posterior_mean_z_max"] < 5.0, res
    lo, hi = res["posterior_sd_ratio_range"]
    assert 0.8 < lo and hi < 1.25, res
    # the delayed-acceptance chains move, and stage 2 runs only on stage-1 survivors
    assert res["da_hmc"]["accept"] > 0.005 and res["da_hmc"]["exact_ll_evals"] > 0
    assert res["da_hmc"]["exact_ll_evals"] <= res["da_iters"] * res["chains"]
