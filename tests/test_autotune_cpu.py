"""Host logic of the plan autotuner: the choice among timed candidates and
the cache key (no GPU)."""
from __future__ import annotations

from paper_2510_11077_gb300 import autotune


def _t(w, c, tape, ms):
    return {"plan": {"walkers_per_cta": w, "ctas_per_sm": c, "tape_cache": tape}, "ms": ms}


def test_pick_prefers_fewest_resident_lanes_among_ties():
    tried = [_t(64, 16, 1, 211.80), _t(32, 8, 1, 211.83), _t(64, 4, 1, 212.15),
             _t(128, 16, 1, 212.26), _t(32, 16, 0, 308.3), {"plan": _t(128, 16, 1, 0)["plan"], "ms": None}]
    assert autotune.pick(tried)["plan"] == {"walkers_per_cta": 32, "ctas_per_sm": 8, "tape_cache": 1}


def test_pick_takes_the_fastest_outside_the_tie_band():
    tried = [_t(32, 4, 0, 100.0), _t(128, 16, 1, 80.0)]
    assert autotune.pick(tried)["ms"] == 80.0
    assert autotune.pick(tried, tie=0.3)["ms"] == 100.0


def test_plan_key_separates_noise_models_and_sources():
    k_rw = autotune.plan_key([10, 20], 64, True, "GPU", "rw")
    k_ou = autotune.plan_key([10, 20], 64, True, "GPU", "ou")
    assert k_rw != k_ou and k_rw.endswith(autotune._source_hash())
