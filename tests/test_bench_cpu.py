"""The bench's reference arm (the oracle on the host cores) keeps the JSON
contract, and its non-zero ranks exit without work.  CPU only."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_prints_one_contract_line():
    out = run_bench("--impl", "reference", "--steps", "2", "--warmup", "1",
                    "--workload", "psr20_toa500-2000_w4096")
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    for k in ("metric", "value", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == "psr20_toa500-2000_w4096"


def test_reference_arm_samples_a_batch_smaller_than_a_step():
    # one walker in the workload's batch: each step still evaluates its full
    # sample (the walker repeated), so the rate counts work actually done
    out = run_bench("--impl", "reference", "--steps", "1", "--warmup", "0",
                    "--workload", "psr1_toa1000")
    d = json.loads([l for l in out.splitlines() if l.startswith("{")][0])
    assert d["value"] > 0 and d["config"]["batch"] == 1


def test_reference_arm_other_ranks_exit_quietly():
    out = run_bench("--impl", "reference", "--steps", "1", "--warmup", "0",
                    env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""
