"""Autotuner of the batched filter's schedule (lane packing and block shape).

A plan fixes how (walker, pulsar) lanes are packed into thread blocks
(walkers_per_cta walkers of one pulsar per block), how many blocks stay
resident per SM in the persistent grid, the adjoint checkpoint stride and
whether the adjoint keeps its tape in HBM.  The tuner times every candidate
with CUDA events on a sub-batch of the caller's walkers, skips candidates
that do not fit in device memory, applies the fastest and records it in a
JSON cache keyed by the array's shape, the batch size, the noise model, the
GPU and the library source, so later runs reuse it without timing.
Candidates within `tie` (relative) of the fastest count as equally fast; of
those the tuner takes the one with the fewest resident lanes (walkers per
block x blocks per SM), whose scratch -- the adjoint tape above all -- takes
the least device memory.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import argus

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuned_plans.json")

TIE = 0.01

DEFAULT_SPACE = {
    "walkers_per_cta": (32, 64, 128),
    "ctas_per_sm": (4, 8, 12, 16),
    "tape_cache": (0, 1),
    "ckpt_stride": (0,),
}


FILTER_SOURCES = ("kf_kernels.cu", "kf_model.cuh", "kf_math.cuh", "kf_internal.cuh")


def source_hash() -> str:
    return _source_hash()


def _source_hash() -> str:
    """Hash of the batched filter kernels' sources: a tuned plan (and a recorded
    ncu traffic figure) is stale once they change."""
    h = hashlib.sha256()
    csrc = os.path.join(HERE, "csrc")
    for f in FILTER_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def plan_key(n_toa, batch: int, grad: bool, gpu_name: str, model: str = "rw") -> str:
    shape = hashlib.sha256(",".join(str(int(n)) for n in n_toa).encode()).hexdigest()[:16]
    return (f"{gpu_name}|P{len(n_toa)}|toa{shape}|B{batch}|{'grad' if grad else 'll'}|{model}"
            f"|src{_source_hash()}")


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_plan(arr, theta, grad: bool, reps: int) -> float:
    import torch
    B = theta.shape[0]
    ll = torch.empty(B, dtype=torch.float64, device=theta.device)
    g = torch.empty((B, arr.dim), dtype=torch.float64, device=theta.device) if grad else None
    call = (lambda: argus.argus_loglik_grad(arr, theta, ll, g)) if grad else \
        (lambda: argus.argus_loglik(arr, theta, ll))
    call()                                   # capture / allocate
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(theta.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def pick(tried: list, tie: float = TIE) -> dict:
    """The chosen entry of a list of timed candidates (see the module note)."""
    ok = [t for t in tried if t.get("ms") is not None]
    fastest = min(t["ms"] for t in ok)
    near = [t for t in ok if t["ms"] <= fastest * (1.0 + tie)]
    return min(near, key=lambda t: (t["plan"]["walkers_per_cta"] * t["plan"]["ctas_per_sm"], t["ms"]))


def autotune(arr, theta, n_toa, grad: bool = True, space: dict | None = None,
             tune_batch: int | None = None, reps: int = 2, cache_path: str | None = DEFAULT_CACHE,
             batch_for_key: int | None = None, log=None, tie: float = TIE) -> dict:
    """Pick the fastest plan for `arr` on walkers `theta` (a CUDA tensor).

    tune_batch: time on the first tune_batch walkers only (default: all).
    Returns {"plan": ..., "ms": ..., "tried": [...], "cached": bool}.
    """
    import torch
    space = dict(DEFAULT_SPACE, **(space or {}))
    B = theta.shape[0] if batch_for_key is None else batch_for_key
    model = argus.model_name(getattr(arr, "model", 0))
    key = plan_key(n_toa, B, grad, torch.cuda.get_device_name(theta.device), model)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache:
        arr.set_plan(**cache[key]["plan"])
        return dict(cache[key], cached=True)
    th = theta[:tune_batch].contiguous() if tune_batch else theta
    tried = []
    names = list(space)
    for values in itertools.product(*(space[k] for k in names)):
        plan = dict(zip(names, values), mode=argus.ARGUS_MODE_BATCHED, use_graph=1)
        try:
            arr.set_plan(**plan)
            ms = _time_plan(arr, th, grad, reps)
        except argus.ArgusError as err:
            if err.status != 3:          # only out-of-memory candidates are skipped
                raise
            tried.append(dict(plan=plan, ms=None, note="out of device memory"))
            continue
        tried.append(dict(plan=plan, ms=ms))
        if log:
            log(f"autotune {plan} -> {ms:.2f} ms")
    if not any(t["ms"] is not None for t in tried):
        raise argus.ArgusError(3, "no candidate plan fits in device memory")
    best = pick(tried, tie)
    arr.set_plan(**best["plan"])
    rec = {"plan": best["plan"], "ms": best["ms"], "tune_batch": th.shape[0], "tried": tried}
    if cache_path:
        src = f"|src{_source_hash()}"
        cache = {k: v for k, v in cache.items() if k.endswith(src)}   # drop stale plans
        cache[key] = rec
        save_cache(cache, cache_path)
    return dict(rec, cached=False)
