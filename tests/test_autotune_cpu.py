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


def test_committed_plan_cache_matches_the_kernel_sources():
    """The tuned plans shipped with the library were timed on the current
    filter sources (every key ends with their hash) and lie in the tuner's
    candidate space, so the bench reads them instead of tuning again."""
    cache = autotune.load_cache(autotune.DEFAULT_CACHE)
    assert cache
    for key, rec in cache.items():
        assert key.endswith("src" + autotune.source_hash()), key
        for field in ("walkers_per_cta", "ctas_per_sm", "tape_cache"):
            assert rec["plan"][field] in autotune.DEFAULT_SPACE[field], (key, field)


def test_recorded_ncu_counts_match_the_kernel_sources():
    """profiles/traffic.json's FP64 instruction and DRAM counts were taken on
    the current filter sources (the bench reports them only then)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                        "traffic.json")
    records = json.load(open(path))
    assert {"k_filter_grad", "k_filter_fwd", "k_filter_grad_ou"} <= set(records)
    for name, rec in records.items():
        assert rec["source_sha"] == autotune.source_hash(), name
