"""The seeded synthetic inputs follow the stated recipe: workload shapes and
TOA counts, sorted TOAs over a 10-year span from the array epoch, unit pulsar
positions, TOA errors, the prior box, parameter layouts and reproducibility.
CPU only; the generator holds none of the likelihood's arithmetic."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2510_11077_gb300 import inputs

# name -> (pulsars, total TOAs, batch)
EXPECT = {
    "psr1_toa1000": (1, 1000, 1),
    "psr20_toa500-2000_w4096": (20, 26182, 4096),
    "psr67_toa5000_w1024": (67, 335000, 1024),
    "psr100_toalognormal_w16384": (100, 449398, 16384),
}


@pytest.mark.parametrize("name", list(EXPECT))
def test_workload_shapes_and_toas(name):
    P, total, B = EXPECT[name]
    d = inputs.make_workload_array(name)
    assert d.n_pulsars == P and int(d.n_toa.sum()) == total and inputs.WORKLOADS[name].batch == B
    assert d.dim == 7 + 2 * P
    assert d.t.min() == 0.0 and d.t.max() <= inputs.T_OBS
    for p in range(P):
        t, r, s = d.pulsar(p)
        assert np.all(np.diff(t) >= 0.0) and np.all(np.isfinite(r))
        assert np.all(s == inputs.SIGMA_TOA)
    assert np.allclose(np.linalg.norm(d.pos, axis=1), 1.0, atol=1e-12)
    assert np.all(d.equad == 0.0) and np.allclose(d.p0, inputs.P0_DEFAULT)
    law = inputs.WORKLOADS[name].toa_law
    if law[0] == "uniform":
        assert d.n_toa.min() >= law[1] and d.n_toa.max() <= law[2]
    if law[0] == "lognormal":
        assert d.n_toa.min() >= law[3] and d.n_toa.max() <= law[4]


def test_workloads_are_reproducible():
    a = inputs.make_workload_array("psr20_toa500-2000_w4096")
    b = inputs.make_workload_array("psr20_toa500-2000_w4096")
    for f in ("off", "t", "r", "sigma", "pos", "theta_true"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    ta = inputs.make_theta_batch(a, 32, seed=5)
    assert np.array_equal(ta, inputs.make_theta_batch(b, 32, seed=5))
    assert not np.array_equal(ta, inputs.make_theta_batch(b, 32, seed=6))


def in_box(theta, box):
    return np.all((theta >= box[:, 0]) & (theta <= box[:, 1]))


@pytest.mark.parametrize("model,pt", [("rw", False), ("ou", False), ("rw", True), ("ou", True)])
def test_parameter_layout_and_prior_box(model, pt):
    d = inputs.make_array(np.array([40, 0, 75]), seed=3, model=model, pulsar_term=pt)
    k = (3 if model == "ou" else 2) + (1 if pt else 0)
    assert d.n_per_pulsar == k and d.dim == 7 + k * 3 and len(d.theta_true) == d.dim
    box = inputs.noise_prior(model, pt)
    prior = inputs.make_theta_batch(d, 500, seed=4, kind="prior")
    assert prior.shape == (500, d.dim)
    assert in_box(prior[:, :7], inputs.PRIOR_GW)
    assert in_box(prior[:, 7:].reshape(-1, k), box)
    post = inputs.make_theta_batch(d, 500, seed=4)
    assert np.all(np.abs(post[:, 3]) <= 1.0) and np.all(np.abs(post[:, 4]) < 1.0)
    assert np.all(post[:, 7 + d.efac_slot::k] > 0.0)
    if pt:
        assert np.all(post[:, 7 + k - 1::k] > 0.0)
        dist = d.theta_true[7 + k - 1::k]
        assert np.all((dist >= inputs.PRIOR_DIST[0, 0]) & (dist <= inputs.PRIOR_DIST[0, 1]))


def test_pulsar_term_flag_leaves_the_residuals_unchanged():
    a = inputs.make_array(np.array([30, 50]), seed=8)
    b = inputs.make_array(np.array([30, 50]), seed=8, pulsar_term=True)
    assert np.array_equal(a.t, b.t) and np.array_equal(a.r, b.r)
