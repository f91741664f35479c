#!/usr/bin/env python
"""Benchmark of the batched FP64 Kalman-filter log-likelihood + gradient.

One step = one evaluation of loglik and its full gradient for a whole batch of
parameter vectors (K1 projection -> K3 checkpointed adjoint filter -> K4
reduction), with the batch's inputs resident in HBM.  Metric: loglik+grad
evaluations (parameter vectors) per second, whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Default workload: 100 pulsars, log-normal TOA counts (median 3000, clipped to
[200, 20000], 449,398 TOAs), 16384 walkers, D = 207, FP64.  Multi-GPU runs
(torchrun) give each rank its own 16384 walkers (weak scaling, no collective
on the data path).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "loglik+grad evals/s on 1 GB300, batched vs plain filter; % FP64/HBM roofline"
UNIT = "evals/s"
DEFAULT_WORKLOAD = "psr100_toalognormal_w16384"
# FP64 peak derived from the part's unit counts and clock: 2 FP64 FMA per
# clock per SM x 2 flop x 152 SMs x 2.07 GHz = 1.2586 TFLOP/s (the nominal
# 1.25 TFLOP/s of a GB300).
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
# Algorithmic FP64 flops per lane-step of the gradient kernel: the forward
# recursion counts 40 flops per TOA (predict 6 FMA + 2 add, signal and
# innovation 4 FMA + 2 add, update 1 rcp + 2 mul + 5 FMA + 2 quad, FMA = 2
# flops, transcendentals not counted); forward + recompute + adjoint = 3x.
FLOPS_PER_LANE_STEP_FWD = 40
FLOPS_PER_LANE_STEP_GRAD = 120
# With Ornstein-Uhlenbeck red noise the forward step also builds F and Q from
# gamma dt: 1 mul for x, a 7-term Horner series (6 FMA, the shortest of the
# kernel's three), 4 FMA of recurrence, 6 flops for phi4, 8 for the
# coefficients and 4 more in the prediction = 39 flops; 79 per lane-step, and
# the gradient counted, as above, as 3x the forward.
FLOPS_PER_LANE_STEP_FWD_OU = 79
FLOPS_PER_LANE_STEP_GRAD_OU = 3 * FLOPS_PER_LANE_STEP_FWD_OU
# FP64 instructions (DFMA + DMUL + DADD, thread-level) per lane-step, counted
# by ncu (profiles/traffic.json, with the source hash they were taken on)
LOGLIK_WORKLOAD = "psr20_toa500-2000_w4096"
PSR67_WORKLOAD = "psr67_toa5000_w1024"
OU_WORKLOAD = "psr20_toa500-2000_w4096"
L2_FLUSH_BYTES = 256 << 20
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--plain-walkers", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-loglik", action="store_true",
                    help="skip the loglik-only leg (20 pulsars x 4096 walkers)")
    ap.add_argument("--no-ou", action="store_true",
                    help="skip the Ornstein-Uhlenbeck red-noise leg (20 pulsars x 4096 walkers)")
    ap.add_argument("--noise", choices=["rw", "ou"], default="rw",
                    help="red-noise model of the main step (rw: random walk; ou: Ornstein-Uhlenbeck)")
    ap.add_argument("--pulsar-term", action="store_true",
                    help="main step with the wave's pulsar term (distance d_p per pulsar)")
    ap.add_argument("--no-pt", action="store_true",
                    help="skip the pulsar-term leg (20 pulsars x 4096 walkers)")
    ap.add_argument("--no-latency", action="store_true",
                    help="skip the single-walker latency leg (1 pulsar x 1000 TOAs)")
    ap.add_argument("--no-gwb", action="store_true",
                    help="skip the Hellings-Downs GW-background leg (20 pulsars, joint filter)")
    ap.add_argument("--gwb-batch", type=int, default=1216,
                    help="parameter vectors of the GW-background leg")
    ap.add_argument("--no-psr67", action="store_true",
                    help="skip the 67-pulsar x 5000-TOA x 1024-walker loglik+grad leg")
    ap.add_argument("--no-da", action="store_true",
                    help="skip the delayed-acceptance HMC leg (surrogate vs exact HMC, 4096 chains)")
    ap.add_argument("--no-fp64-probe", action="store_true",
                    help="skip the measured FP64 FMA-rate leg")
    ap.add_argument("--autotune", choices=["cache", "off", "force"], default="cache",
                    help="cache: use the tuned-plan cache, tuning on a miss; force: retune")
    ap.add_argument("--tune-batch", type=int, default=4096)
    ap.add_argument("--mode", choices=["filter", "da-hmc", "surrogate", "latency", "gwb"], default="filter",
                    help="filter: loglik+grad evals/s (default); da-hmc: surrogate delayed acceptance; "
                         "surrogate: the surrogate's evaluation alone, fused vs per-layer; "
                         "latency: the single-vector latency leg alone (sequential vs time-parallel); "
                         "gwb: the Hellings-Downs GW-background leg alone (joint filter, --gwb-batch vectors)")
    ap.add_argument("--latency-reps", type=int, default=200,
                    help="timed calls per path in the latency leg")
    ap.add_argument("--plan", default="",
                    help="fixed plan, e.g. tape_cache=1,walkers_per_cta=128 (disables autotune)")
    return ap.parse_args()


def dist_env():
    from paper_2510_11077_gb300 import dist as pdist
    return pdist.env()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), max=float(f[2]), reasons=f[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = sorted({n for r in rows for n, v in zip(names, r["reasons"][1:]) if v == "Active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": seen, "samples": len(rows)}


def traffic_record(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source is unchanged since the counters were taken; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    from paper_2510_11077_gb300 import autotune
    return rec if rec.get("source_sha") == autotune.source_hash() else None


def fp64_rate(local, iters=65536, launches=3):
    """Measured FP64 FMA issue rate of this GPU (argus_selftest_dfma_rate:
    independent FMA chains, 2048 threads per SM; four operand and chain
    variants, the fastest taken), with nvidia-smi clocks sampled while it
    runs.  Returns the best variant's median launch in FMA/s and the FLOP/s
    peak it implies (2 flop per FMA)."""
    import ctypes

    from paper_2510_11077_gb300 import argus
    lib = argus.load()
    lib.argus_selftest_dfma_rate.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.c_void_p]
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clocks = ClockSampler(vis.split(",")[local] if vis else str(local))
    clocks.start()
    time.sleep(0.3)
    names = ["8 chains, parameter operands", "8 chains, register operands", "4 chains",
             "16 chains"]
    variants = {}
    for v, name in enumerate(names):
        rate = (ctypes.c_double * launches)()
        ms = (ctypes.c_float * launches)()
        st = lib.argus_selftest_dfma_rate(iters, launches, v, rate, ms)
        if st != 0:
            clocks.stop()
            raise RuntimeError(f"argus_selftest_dfma_rate failed with status {st}")
        variants[name] = {"fma_per_s": statistics.median(rate), "launch_ms": list(ms)}
    clk = clocks.stop()
    best = max(variants, key=lambda k: variants[k]["fma_per_s"])
    med = variants[best]["fma_per_s"]
    n_sm = None
    try:
        import torch
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    except Exception:
        pass
    out = {"fma_per_s": med, "tflops": 2 * med / 1e12, "best_variant": best, "variants": variants,
           "clocks": clk,
           "how": f"{launches} launches per variant, 8 x {iters} FMAs per thread, 2048 threads "
                  f"per SM (CUDA events, median launch of the fastest variant)"}
    if clk and n_sm:
        out["fma_per_clk_per_sm"] = med / (n_sm * clk["sm_mhz"] * 1e6)
    return out


def _oracle_rate(data, theta, threads, seconds):
    from oracle import kalman
    used = kalman.set_threads(threads)
    done, t0, i = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < seconds:
        rows = theta[i % len(theta): i % len(theta) + used]
        kalman.loglik_grad(data, rows)
        done += len(rows)
        i += used
    dt = time.perf_counter() - t0
    return done / dt, done, dt, used


def dense_vs_kalman():
    """The O(N^3) dense multivariate normal (Cholesky) against the O(N)
    filter, one pulsar, one parameter vector, on this host (the oracle's own
    implementations of each)."""
    import numpy as np

    from oracle import dense, kalman
    from paper_2510_11077_gb300 import inputs
    kalman.set_threads(1)
    out = []
    for n in (250, 500, 1000, 2000):
        d = inputs.make_array(np.array([n]), seed=n)
        th = inputs.make_theta_batch(d, 1, seed=1)
        row = {"toas": n}
        for name, f in (("dense_s", lambda: dense.loglik(d, th)), ("kalman_s", lambda: kalman.loglik(d, th))):
            f()
            t0 = time.perf_counter()
            reps = 0
            while time.perf_counter() - t0 < 0.3:
                f(); reps += 1
            row[name] = (time.perf_counter() - t0) / reps
        out.append(row)
    return out


def cpu_baseline(data, theta, seconds):
    """The CPU oracle as it stands on this host's cores, on a bounded sample:
    all cores (OpenMP over walkers) and one core."""
    cores = os.cpu_count() or 1
    v_all, done, dt, used = _oracle_rate(data, theta, cores, seconds)
    v_one, done1, dt1, _ = _oracle_rate(data, theta, 1, max(2.0, seconds / 3))
    return {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "single_core": {"value": v_one, "unit": UNIT, "sample": f"{done1} walkers, {dt1:.1f} s"},
            "dense_vs_kalman_1psr": dense_vs_kalman(),
            "sample": f"{done} walkers of the same workload (complex-step gradient, OpenMP over "
                      f"walkers), {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    from oracle import kalman
    from paper_2510_11077_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    data = inputs.make_workload_array(w.name, model=args.noise, pulsar_term=args.pulsar_term)
    theta = inputs.make_theta_batch(data, w.batch, seed=w.seed)
    cores = os.cpu_count() or 1
    kalman.set_threads(cores)
    per_step = cores * 2

    def sample(i):   # step i's walkers, wrapping around a batch smaller than the sample
        return theta[(i * per_step + np.arange(per_step)) % len(theta)]

    for i in range(args.warmup):
        kalman.loglik_grad(data, sample(i))
    t0 = time.perf_counter()
    for i in range(args.steps):
        kalman.loglik_grad(data, sample(i))
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name + ("" if args.noise == "rw" else " (OU red noise)")
                                   + (" (with pulsar term)" if args.pulsar_term else ""),
                       "pulsars": data.n_pulsars, "toas": int(data.n_toa.sum()),
                       "batch": w.batch, "dim": data.dim,
                       "step": f"{per_step} walkers of the batch per step (bounded CPU sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} walkers per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def loglik_only(args, dev, local, fp64=None):
    """Forward filter alone (K1 -> K2 -> K4) on the 20-pulsar, 4096-walker array:
    loglik evals/s with the forward kernel timed live and its FP64 roofline."""
    import torch

    from paper_2510_11077_gb300 import argus, autotune, inputs
    w = inputs.WORKLOADS[LOGLIK_WORKLOAD]
    data = inputs.make_workload_array(w.name)
    theta = torch.from_numpy(inputs.make_theta_batch(data, w.batch, seed=w.seed)).to(dev)
    theta_prior = torch.from_numpy(inputs.make_theta_batch(data, w.batch, seed=w.seed + 7,
                                                           kind="prior")).to(dev)
    arr = argus.Array(data, device=local)
    res = autotune.autotune(arr, theta, data.n_toa, grad=False, batch_for_key=w.batch,
                            space={"tape_cache": (0,)})
    ll = torch.empty(w.batch, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    arr.set_timing(True)
    for _ in range(3):
        argus.argus_loglik(arr, theta, ll)
    torch.cuda.synchronize(dev)
    reps = 20
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    kern = []
    for k in range(reps):
        flush.zero_()
        ev[k][0].record(stream)
        argus.argus_loglik(arr, theta, ll)
        ev[k][1].record(stream)
        kern.append(arr.get_timing()[1])
    torch.cuda.synchronize(dev)
    step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    k_ms = statistics.mean(kern)
    # the same batch size drawn from the prior: the path does not depend on the values
    llp = torch.empty(w.batch, dtype=torch.float64, device=dev)
    argus.argus_loglik(arr, theta_prior, llp)
    torch.cuda.synchronize(dev)
    evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        flush.zero_()
        evp[k][0].record(stream)
        argus.argus_loglik(arr, theta_prior, llp)
        evp[k][1].record(stream)
    torch.cuda.synchronize(dev)
    prior_ms = statistics.mean(a.elapsed_time(b) for a, b in evp)
    lane_steps = w.batch * int(data.n_toa.sum())
    arr.close()
    return {"workload": w.name, "metric": "loglik evals/s", "value": w.batch / (step_ms * 1e-3),
            "ms_per_step": step_ms, "prior_draws_ms_per_step": prior_ms,
            "lane_steps_per_s": lane_steps / (step_ms * 1e-3),
            "plan": res["plan"], "autotune_cached": res["cached"],
            "roofline": fp64_roofline("k_filter_fwd", FLOPS_PER_LANE_STEP_FWD, lane_steps, k_ms,
                                      fp64)}


def ou_leg(args, dev, local, fp64=None):
    """Loglik + gradient with Ornstein-Uhlenbeck red noise (D = 7 + 3P) on the
    20-pulsar, 4096-walker array: evals/s, the adjoint kernel timed live and
    its FP64 roofline."""
    import torch

    from paper_2510_11077_gb300 import argus, autotune, inputs
    w = inputs.WORKLOADS[OU_WORKLOAD]
    data = inputs.make_workload_array(w.name, model="ou")
    theta = torch.from_numpy(inputs.make_theta_batch(data, w.batch, seed=w.seed)).to(dev)
    arr = argus.Array(data, device=local)
    res = autotune.autotune(arr, theta, data.n_toa, grad=True, batch_for_key=w.batch)
    ll = torch.empty(w.batch, dtype=torch.float64, device=dev)
    g = torch.empty((w.batch, data.dim), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    arr.set_timing(True)
    for _ in range(3):
        argus.argus_loglik_grad(arr, theta, ll, g)
    torch.cuda.synchronize(dev)
    reps = 10
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    kern = []
    for k in range(reps):
        flush.zero_()
        ev[k][0].record(stream)
        argus.argus_loglik_grad(arr, theta, ll, g)
        ev[k][1].record(stream)
        kern.append(arr.get_timing()[1])
    torch.cuda.synchronize(dev)
    step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    k_ms = statistics.mean(kern)
    lane_steps = w.batch * int(data.n_toa.sum())
    arr.close()
    return {"workload": w.name + " (Ornstein-Uhlenbeck red noise)", "dim": data.dim,
            "metric": "loglik+grad evals/s", "value": w.batch / (step_ms * 1e-3),
            "ms_per_step": step_ms, "plan": res["plan"], "autotune_cached": res["cached"],
            "roofline": fp64_roofline("k_filter_grad_ou", FLOPS_PER_LANE_STEP_GRAD_OU, lane_steps,
                                      k_ms, fp64, traffic=bool(res["plan"].get("tape_cache")))}


def psr67_leg(args, dev, local, fp64=None):
    """Loglik + full gradient (7 GW + 2 noise parameters per pulsar, D = 141)
    on the 67-pulsar array with 5000 TOAs each and 1024 walkers, through the
    adjoint kernel with its own autotuned plan: evals/s, the kernel timed live
    and its FP64 roofline."""
    import torch

    from paper_2510_11077_gb300 import argus, autotune, inputs
    w = inputs.WORKLOADS[PSR67_WORKLOAD]
    data = inputs.make_workload_array(w.name)
    theta = torch.from_numpy(inputs.make_theta_batch(data, w.batch, seed=w.seed)).to(dev)
    arr = argus.Array(data, device=local)
    res = autotune.autotune(arr, theta, data.n_toa, grad=True, batch_for_key=w.batch)
    ll = torch.empty(w.batch, dtype=torch.float64, device=dev)
    g = torch.empty((w.batch, data.dim), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    arr.set_timing(True)
    for _ in range(3):
        argus.argus_loglik_grad(arr, theta, ll, g)
    torch.cuda.synchronize(dev)
    reps = 10
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    kern = []
    for k in range(reps):
        flush.zero_()
        ev[k][0].record(stream)
        argus.argus_loglik_grad(arr, theta, ll, g)
        ev[k][1].record(stream)
        kern.append(arr.get_timing()[1])
    torch.cuda.synchronize(dev)
    finite = bool(torch.isfinite(ll).all().item() and torch.isfinite(g).all().item())
    arr.close()
    step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    k_ms = statistics.mean(kern)
    lane_steps = w.batch * int(data.n_toa.sum())
    roof = fp64_roofline("k_filter_grad", FLOPS_PER_LANE_STEP_GRAD, lane_steps, k_ms, fp64)
    return {"workload": w.name, "dim": data.dim, "metric": "loglik+grad evals/s",
            "value": w.batch / (step_ms * 1e-3), "unit": UNIT, "ms_per_step": step_ms,
            "lane_steps_per_s": lane_steps / (step_ms * 1e-3), "finite": finite,
            "plan": res["plan"], "autotune_cached": res["cached"],
            "l2": "flushed between timed steps (256 MiB write, untimed)", "roofline": roof}


def fp64_roofline(kernel, flops_per_lane_step, lane_steps, kernel_ms, fp64=None, traffic=True):
    """FP64 roofline of one filter launch.  achieved: the algorithmic count
    (flops_per_lane_step x lane-steps) per event-timed launch; peak: the
    2 FMA/clk/SM x 152 SMs x 2.07 GHz derived peak; peak_measured and
    frac_measured: against this run's measured FP64 FMA rate (fp64_rate);
    fp64_issue_frac: the FP64 instructions the kernel executes per lane-step
    (ncu count in profiles/traffic.json, taken on the same kernel source) per
    second, over the measured FMA issue rate -- the FP64 pipe's busy share."""
    achieved = flops_per_lane_step * lane_steps / (kernel_ms * 1e-3) / 1e12
    tr = traffic_record(kernel)
    out = {"bound": "alu", "kernel": kernel, "kernel_ms": kernel_ms, "achieved": achieved,
           "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
           "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz",
           "algorithmic": f"{flops_per_lane_step} FP64 flop per lane-step x {lane_steps} "
                          f"lane-steps per launch",
           "traffic": (tr["dram_bytes_per_lane_step"] * lane_steps
                       if tr and traffic and tr.get("dram_bytes_per_lane_step") else None)}
    if fp64:
        out["peak_measured"] = fp64["tflops"]
        out["frac_measured"] = achieved / fp64["tflops"]
        out["peak_measured_source"] = "argus_selftest_dfma_rate in this run (median launch)"
    instr = tr.get("fp64_instr_per_lane_step") if tr else None
    if instr:
        rate = instr * lane_steps / (kernel_ms * 1e-3)
        out["fp64_instr_per_lane_step"] = instr
        out["fp64_instr_per_s"] = rate
        if fp64:
            out["fp64_issue_frac"] = rate / fp64["fma_per_s"]
        out["fp64_issue_frac_derived"] = rate / (FP64_PEAK_TFLOPS * 1e12 / 2)
    return out


def pulsar_term_leg(args, dev, local):
    """Loglik + gradient with the wave's pulsar term on the 20-pulsar,
    4096-walker array, against the same array without it: the filter kernels
    are shared, so the leg reports the stage times of K1 (projection, where the
    pulsar term is folded in) and K4 (reduction, its chain rule)."""
    import torch

    from paper_2510_11077_gb300 import argus, autotune, inputs
    w = inputs.WORKLOADS[OU_WORKLOAD]
    out = {}
    for pt in (False, True):
        data = inputs.make_workload_array(w.name, pulsar_term=pt)
        theta = torch.from_numpy(inputs.make_theta_batch(data, w.batch, seed=w.seed)).to(dev)
        arr = argus.Array(data, device=local)
        res = autotune.autotune(arr, theta, data.n_toa, grad=True, batch_for_key=w.batch)
        ll = torch.empty(w.batch, dtype=torch.float64, device=dev)
        g = torch.empty((w.batch, data.dim), dtype=torch.float64, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream(dev)
        arr.set_timing(True)
        for _ in range(3):
            argus.argus_loglik_grad(arr, theta, ll, g)
        torch.cuda.synchronize(dev)
        reps = 10
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        stages = []
        for k in range(reps):
            flush.zero_()
            ev[k][0].record(stream)
            argus.argus_loglik_grad(arr, theta, ll, g)
            ev[k][1].record(stream)
            stages.append(arr.get_timing())
        torch.cuda.synchronize(dev)
        step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        arr.close()
        out["with_pulsar_term" if pt else "earth_term_only"] = {
            "dim": data.dim, "value": w.batch / (step_ms * 1e-3), "unit": UNIT,
            "ms_per_step": step_ms, "plan": res["plan"],
            "stage_ms": {"project": statistics.mean(x[0] for x in stages),
                         "filter": statistics.mean(x[1] for x in stages),
                         "reduce": statistics.mean(x[2] for x in stages)}}
    out["workload"] = w.name
    out["metric"] = "loglik+grad evals/s"
    return out


LATENCY_WORKLOAD = "psr1_toa1000"


def gwb_flops_per_toa(P: int) -> int:
    """Algorithmic FP64 flops of one TOA of the joint filter in the scaled
    frame that k_gwb_filter runs (FMA = 2).  The decays are carried in scale
    factors, so the transition is the identity but for each pulsar's rho row.
    The predict of an upper 3x3 block then changes only its rho row and
    column: 12 FMA for (Fh X Fh^T) and 4 for the GW process noise, 32 flops
    (a diagonal block: 8 + 4 FMA and 3 adds, 25).  Per pulsar the mean
    predict costs 4.  The update costs 1 FMA per upper entry of the 3P x 3P
    covariance, n multiplies for c/S and n FMA for the mean.  The textbook
    unscaled filter takes 44 flops per block and 3 per upper entry
    (gwb_flops_per_toa_unscaled)."""
    n = 3 * P
    return 32 * P * (P - 1) // 2 + 25 * P + 4 * P + n + n * (n + 1) + 2 * n


def gwb_flops_per_toa_unscaled(P: int) -> int:
    """FP64 flops of one TOA of the textbook joint filter: the predict of each
    upper 3x3 block (F_I X: 18, (F_I X) F_J^T: 18, Q: 8), the symmetric
    rank-1 update (3 per upper entry) and the mean (10 per pulsar)."""
    n = 3 * P
    return 44 * P * (P + 1) // 2 + 3 * n * (n + 1) // 2 + 10 * P


def gwb_leg(args, dev, local):
    """Joint likelihood with a Hellings-Downs correlated GW background on the
    20-pulsar array (26,182 TOAs, 60-dimensional joint state): evals/s with
    --gwb-batch parameter vectors, and the FP64 roofline of the joint filter."""
    import numpy as np
    import torch

    from paper_2510_11077_gb300 import argus, inputs
    w = inputs.WORKLOADS[LOGLIK_WORKLOAD]
    data = inputs.make_workload_array(w.name)
    P = data.n_pulsars
    GWB_BATCH = args.gwb_batch
    rng = np.random.default_rng(w.seed)
    th = np.empty((GWB_BATCH, 2 + 3 * P))
    th[:, 0] = rng.uniform(-20.0, -18.5, GWB_BATCH)
    th[:, 1] = rng.uniform(-9.5, -7.5, GWB_BATCH)
    th[:, 2::3] = rng.uniform(-20.8, -19.2, (GWB_BATCH, P))
    th[:, 3::3] = rng.uniform(-9.8, -7.2, (GWB_BATCH, P))
    th[:, 4::3] = rng.uniform(0.85, 1.15, (GWB_BATCH, P))
    theta = torch.from_numpy(th).to(dev)
    arr = argus.GwbArray(data, device=local)
    ll = torch.empty(GWB_BATCH, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    argus.argus_gwb_loglik(arr, theta, ll)
    torch.cuda.synchronize(dev)
    reps = 3
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        argus.argus_gwb_loglik(arr, theta, ll)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    # the same batch with the gradient (reverse-mode adjoint through the joint filter)
    g = torch.empty((GWB_BATCH, 2 + 3 * P), dtype=torch.float64, device=dev)
    argus.argus_gwb_loglik_grad(arr, theta, ll, g)
    torch.cuda.synchronize(dev)
    gms = []
    for _ in range(2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        argus.argus_gwb_loglik_grad(arr, theta, ll, g)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        gms.append(e0.elapsed_time(e1))
    grad_finite = bool(torch.isfinite(g).all().item())
    arr.close()
    step_ms = statistics.mean(ms)
    grad_ms = statistics.mean(gms)
    n_toa = int(data.n_toa.sum())
    flops = gwb_flops_per_toa(P) * n_toa * GWB_BATCH
    achieved = flops / (step_ms * 1e-3) / 1e12
    return {"workload": w.name + " (joint filter, Hellings-Downs GW background)", "dim": 2 + 3 * P,
            "state_dim": 3 * P, "batch": GWB_BATCH, "metric": "loglik evals/s",
            "value": GWB_BATCH / (step_ms * 1e-3), "ms_per_step": step_ms,
            "finite": bool(torch.isfinite(ll).all().item()),
            "gradient": {"metric": "loglik+grad evals/s", "value": GWB_BATCH / (grad_ms * 1e-3),
                         "ms_per_step": grad_ms, "over_loglik": grad_ms / step_ms,
                         "finite": grad_finite},
            "roofline": {"bound": "alu", "kernel": "k_gwb_filter", "kernel_ms": step_ms,
                         "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS,
                         "algorithmic": f"{gwb_flops_per_toa(P)} FP64 flop per TOA per parameter vector "
                                        f"(scaled frame) x {n_toa} TOAs x {GWB_BATCH}",
                         "textbook_flop_rate": gwb_flops_per_toa_unscaled(P) * n_toa * GWB_BATCH
                         / (step_ms * 1e-3) / 1e12}}


def latency_leg(args, dev, local):
    """Latency of one evaluation of one parameter vector on the 1-pulsar,
    1000-TOA array: the sequential filter (one lane, one thread stepping
    through the TOAs) against the time-parallel filter (plan mode SCAN), for
    the log-likelihood and for the log-likelihood with its gradient (the
    sequential adjoint against the time-parallel one).  Each call is a
    CUDA-graph replay; L2 is flushed before each call, outside the events."""
    import numpy as np
    import torch

    from paper_2510_11077_gb300 import argus, inputs
    w = inputs.WORKLOADS[LATENCY_WORKLOAD]
    data = inputs.make_workload_array(w.name)
    theta = torch.from_numpy(inputs.make_theta_batch(data, 1, seed=w.seed)).to(dev)
    ll = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty((1, data.dim), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": w.name, "metric": "loglik latency", "unit": "us", "walkers": 1}
    plans = (("sequential", dict(mode=argus.ARGUS_MODE_BATCHED, walkers_per_cta=32)),
             ("scan", dict(mode=argus.ARGUS_MODE_SCAN)))

    def timed(arr, call):
        arr.set_timing(True)
        for _ in range(5):
            call()
        torch.cuda.synchronize(dev)
        stages = arr.get_timing()
        arr.set_timing(False)
        for _ in range(3):
            call()                                  # re-capture without the stage events
        torch.cuda.synchronize(dev)
        reps = max(1, getattr(args, "latency_reps", 200))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for k in range(reps):
            flush.zero_()
            ev[k][0].record(stream)
            call()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        us = sorted(a.elapsed_time(b) * 1e3 for a, b in ev)
        return {"median_us": us[reps // 2], "p10_us": us[reps // 10], "p90_us": us[9 * reps // 10],
                "plan": arr.get_plan(),
                "stage_us": {"project": stages[0] * 1e3, "filter": stages[1] * 1e3,
                             "reduce": stages[2] * 1e3}}

    vals, grads = {}, {}
    out["gradient"] = {"metric": "loglik+grad latency", "unit": "us"}
    for name, plan in plans:
        arr = argus.Array(data, device=local)
        arr.set_plan(**plan)
        out[name] = timed(arr, lambda: argus.argus_loglik(arr, theta, ll))
        vals[name] = float(ll.item())
        out["gradient"][name] = timed(arr, lambda: argus.argus_loglik_grad(arr, theta, ll, g))
        grads[name] = g.cpu().numpy()[0].copy()
        arr.close()
    if vals["sequential"] != vals["scan"] and abs(vals["sequential"] - vals["scan"]) > \
            1e-12 * abs(vals["sequential"]):
        raise RuntimeError("scan and sequential filters disagree")
    gs, gp = grads["sequential"], grads["scan"]
    scale = np.maximum(np.abs(gs), 1e-3 * np.abs(gs).max())
    gdiff = float(np.max(np.abs(gp - gs) / scale))
    if not gdiff <= 1e-8:
        raise RuntimeError(f"scan and sequential adjoints disagree ({gdiff:.2e})")
    out["speedup"] = out["sequential"]["median_us"] / out["scan"]["median_us"]
    out["gradient"]["speedup"] = out["gradient"]["sequential"]["median_us"] / \
        out["gradient"]["scan"]["median_us"]
    out["gradient"]["max_rel_diff"] = gdiff
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_2510_11077_gb300 import argus, inputs
    from paper_2510_11077_gb300 import dist as pdist

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.WORKLOADS[args.workload]
    data = inputs.make_workload_array(w.name, model=args.noise, pulsar_term=args.pulsar_term)
    B, D = w.batch, data.dim
    theta_np = inputs.make_theta_batch(data, B, seed=pdist.rank_seed(w.seed, rank))
    theta = torch.from_numpy(theta_np).to(dev)
    arr = argus.Array(data, device=local)
    tuned = None
    if args.plan:
        arr.set_plan(**{k: int(v) for k, v in (kv.split("=") for kv in args.plan.split(","))})
    elif args.autotune != "off":
        from paper_2510_11077_gb300 import autotune
        cache = autotune.DEFAULT_CACHE
        if args.autotune == "force" and os.path.exists(cache):
            c = autotune.load_cache(cache)
            name = args.noise + ("+pt" if args.pulsar_term else "")
            c.pop(autotune.plan_key(data.n_toa, B, True, torch.cuda.get_device_name(dev), name), None)
            autotune.save_cache(c, cache)
        res = autotune.autotune(arr, theta, data.n_toa, grad=True, tune_batch=args.tune_batch,
                                batch_for_key=B)
        tuned = {"cached": res["cached"], "tune_batch": res.get("tune_batch"),
                 "candidates": len(res.get("tried", []))}
    plan = arr.get_plan()
    ll = torch.empty(B, dtype=torch.float64, device=dev)
    g = torch.empty((B, D), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    kern = []

    def step(timed):
        if not timed:
            argus.argus_loglik_grad(arr, theta, ll, g)
            return None
        flush.zero_()                       # evict L2 between timed steps (not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        argus.argus_loglik_grad(arr, theta, ll, g)
        e1.record(stream)
        kern.append(arr.get_timing())
        return e0, e1

    arr.set_timing(True)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gpu_index = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(gpu_index) if rank == 0 else None

    def start_clocks():
        if clocks:
            clocks.start()
            time.sleep(0.3)

    step_s, total_s = pdist.timed_steps(
        step, args.steps, args.warmup, sync=lambda: torch.cuda.synchronize(dev),
        resolve=lambda evs: [a.elapsed_time(b) / 1e3 for a, b in evs], on_start=start_clocks,
        device=dev)
    clk = clocks.stop() if clocks else None
    total_ms = total_s * 1e3
    value = pdist.job_throughput(B * args.steps, world, total_s)
    filt_ms = statistics.mean(k[1] for k in kern)

    # end to end through the public call with pinned host buffers
    e2e = None
    if not args.no_e2e:
        th_h = torch.from_numpy(theta_np).pin_memory()
        ll_h = torch.empty(B, dtype=torch.float64).pin_memory()
        g_h = torch.empty((B, D), dtype=torch.float64).pin_memory()
        arr.set_timing(False)
        argus.argus_loglik_grad(arr, th_h, ll_h, g_h)      # capture the staged graph
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            argus.argus_loglik_grad(arr, th_h, ll_h, g_h)   # H2D, compute, D2H, sync
        e2e_s = pdist.max_over_ranks(time.perf_counter() - t0, device=dev)
        e2e = {"value": pdist.job_throughput(B * args.steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": B * D * 8, "d2h_bytes_per_step": B * 8 + B * D * 8}
        if not np.allclose(ll_h.numpy(), ll.cpu().numpy(), rtol=0, atol=0, equal_nan=True):
            raise RuntimeError("host-buffer path disagrees with the device path")

    arr.close()                   # frees the adjoint tape before the other legs
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # the same math launched once per parameter vector, on a sample of walkers
    n_plain = min(args.plain_walkers, B)
    arr_p = argus.Array(data, device=local)
    arr_p.set_plan(mode=argus.ARGUS_MODE_PLAIN)
    th_p = theta[:n_plain].contiguous()
    llp = torch.empty(n_plain, dtype=torch.float64, device=dev)
    gp = torch.empty((n_plain, D), dtype=torch.float64, device=dev)
    argus.argus_loglik_grad(arr_p, th_p[:2].contiguous(), llp[:2], gp[:2])
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    argus.argus_loglik_grad(arr_p, th_p, llp, gp)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain = {"value": n_plain / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
             "lane_steps_per_s": n_plain * int(data.n_toa.sum()) / (e0.elapsed_time(e1) / 1e3),
             "sample_walkers": n_plain, "launches_per_walker": 3}
    if not torch.equal(llp, ll[:n_plain]):
        raise RuntimeError("plain and batched filters disagree")
    arr_p.close()

    fp64 = None if args.no_fp64_probe else fp64_rate(local)
    loglik_leg = None if args.no_loglik else loglik_only(args, dev, local, fp64)
    ou = None if args.no_ou else ou_leg(args, dev, local, fp64)
    pt_leg = None if args.no_pt else pulsar_term_leg(args, dev, local)
    lat = None if args.no_latency else latency_leg(args, dev, local)
    gwb_l = None if args.no_gwb else gwb_leg(args, dev, local)
    p67 = None if args.no_psr67 else psr67_leg(args, dev, local, fp64)
    lane_steps = B * int(data.n_toa.sum())
    flops = FLOPS_PER_LANE_STEP_GRAD_OU if args.noise == "ou" else FLOPS_PER_LANE_STEP_GRAD
    kname = "k_filter_grad_ou" if args.noise == "ou" else "k_filter_grad"
    roofline = fp64_roofline(kname, flops, lane_steps, filt_ms, fp64,
                             traffic=bool(plan.get("tape_cache")) and not args.pulsar_term)
    peaks, peaks_src = _measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    dram_gbs = roofline["traffic"] / (filt_ms * 1e-3) / 1e9 if roofline["traffic"] else None
    roofline["dram"] = {"achieved_gbs": dram_gbs, "peak_gbs": hbm,
                        "frac": (dram_gbs / hbm) if (dram_gbs and hbm) else None,
                        "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peaks_src})"}
    roofline["headline"] = ("fp64_issue_frac: the FP64 pipe's busy share against the measured FMA "
                            "rate; frac (the algorithmic count over the derived peak) is kept for "
                            "the contract's definition")
    da = None
    if world == 1 and not args.no_da:
        da = da_hmc_leg(local)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(data, theta_np, args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name + ("" if args.noise == "rw" else " (OU red noise)")
                                   + (" (with pulsar term)" if args.pulsar_term else ""),
                       "pulsars": data.n_pulsars,
                       "toas": int(data.n_toa.sum()), "batch_per_gpu": B, "dim": D,
                       "lane_steps_per_gpu": lane_steps, "plan": plan, "autotune": tuned,
                       "l2": "flushed between timed steps (256 MiB write, untimed)"},
            "e2e": e2e, "gpu_launches": 3 * args.steps, "roofline": roofline,
            "lane_steps_per_s": lane_steps * world * args.steps / (total_ms * 1e-3),
            "plain_filter": plain, "batched_over_plain": value / world / plain["value"],
            "stage_ms": {"project": statistics.mean(k[0] for k in kern), "filter": filt_ms,
                         "reduce": statistics.mean(k[2] for k in kern)},
            "clocks": clk, "cpu_baseline": cpu, "loglik_only": loglik_leg,
            "ou_red_noise": ou, "pulsar_term": pt_leg, "latency_1psr": lat, "gwb_hd": gwb_l,
            "psr67_grad": p67, "fp64_peak": fp64, "da_hmc": da}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0}, "fallback"


DA_CONFIG = dict(n_chains=4096, n_train=1_000_000, warmup_iter=200, sample_iter=100, da_iter=400,
                 n_steps=16, epochs=60, batch=4096, lr=1e-3, value_weight=10.0)


def da_hmc_leg(local):
    """Delayed-acceptance HMC with the surrogate (trained on the GPU on 1e6
    exact-filter evaluations) against plain exact-filter HMC, both from the
    same warmed-up state, on the 20-pulsar array with 4096 chains (the
    configuration of `--mode da-hmc`): min-ESS/s of each, the gain with and
    without the surrogate's data generation and training, and the posterior
    agreement (the exact filter is stage 2, so the posterior is unchanged)."""
    from paper_2510_11077_gb300 import da_experiment
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clocks = ClockSampler(vis.split(",")[local] if vis else str(local))
    clocks.start()
    res = da_experiment.run(device=local, **DA_CONFIG)
    clk = clocks.stop()
    h, d = res["hmc"], res["da_hmc"]
    return {"workload": "psr20_toa500-2000_w4096 TOAs with an injected model source, D = 47",
            "chains": res["chains"], "leapfrog_steps": res["leapfrog_steps"],
            "train_rows": res["train_rows"], "epochs": res["epochs"],
            "exact_hmc": {"min_ess_per_s": h["ess_per_s"], "ess_min": h["ess_min"],
                          "seconds": h["seconds"], "iters": res["sample_iters"],
                          "accept": h["accept"], "exact_grad_evals": h["exact_grad_evals"]},
            "da_hmc": {"min_ess_per_s": d["ess_per_s"], "ess_min": d["ess_min"],
                       "seconds": d["seconds"], "iters": res["da_iters"],
                       "accept_stage1": d["accept_stage1"], "accept": d["accept"],
                       "exact_ll_evals": d["exact_ll_evals"],
                       "min_ess_per_s_incl_training": d["ess_per_s_incl_training"]},
            "ess_per_s_gain": res["ess_per_s_gain"],
            "ess_per_s_gain_incl_training": res["ess_per_s_gain_incl_training"],
            "ess_per_exact_eval_gain": (d["ess_min"] / max(d["exact_ll_evals"], 1)) /
                                       (h["ess_min"] / max(h["exact_grad_evals"], 1)),
            "data_gen_s": res["data_gen_s"], "train_s": res["train_s"],
            "posterior_mean_z_max": res["posterior_mean_z_max"],
            "posterior_sd_ratio_range": res["posterior_sd_ratio_range"],
            "holdout_abs_err_nats_median": res["holdout_abs_err_nats_median"],
            "clocks": clk, "experiment": res}


def run_da_hmc(args):
    """Surrogate-accelerated delayed-acceptance HMC on the 20-pulsar array with
    4096 chains, against plain exact HMC; plus the surrogate network's own
    tensor-core throughput."""
    import torch

    from paper_2510_11077_gb300 import surrogate
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    leg = da_hmc_leg(local)
    res = leg["experiment"]
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local]
                          if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local))
    clocks.start()
    # tensor-core throughput of the surrogate: eval of 4096 rows, and a train step
    dev = torch.device("cuda", local)
    net = surrogate.Surrogate(device=local, max_rows=4096, seed=1)
    x = torch.randn((4096, 47), dtype=torch.float32, device=dev)
    ll = torch.randn(4096, dtype=torch.float32, device=dev)
    g = torch.randn((4096, 47), dtype=torch.float32, device=dev)
    for _ in range(5):
        net.eval(x)
        net.train_step(x, ll, g, 1e-4)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    reps = 50
    e[0].record()
    for _ in range(reps):
        net.eval(x)
    e[1].record()
    for _ in range(reps):
        net.train_step(x, ll, g, 1e-4)
    e[2].record()
    # the sampler's mode: value output and its back-propagated input gradient
    net.set_grad_mode(1)
    for _ in range(5):
        net.eval(x)
    e[3].record()
    for _ in range(reps):
        net.eval(x)
    e4 = torch.cuda.Event(enable_timing=True)
    e4.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    eval_ms = e[0].elapsed_time(e[1]) / reps
    train_ms = e[1].elapsed_time(e[2]) / reps
    bp_ms = e[3].elapsed_time(e4) / reps
    layer_macs = 64 * 256 + 3 * 256 * 256 + 256 * 64          # padded shapes
    eval_flop = 2 * layer_macs * 4096
    train_flop = 3 * eval_flop - 2 * 64 * 256 * 4096           # fwd + dX (no dX0) + dW
    bp_flop = eval_flop + 2 * (3 * 256 * 256 + 256 * 64) * 4096  # fwd + back to the input
    peaks, src = _measured_peaks()
    peak = peaks["bf16_tflops"]
    achieved = eval_flop / (eval_ms * 1e-3) / 1e12
    line = {"metric": "effective samples/s: delayed-acceptance HMC with the BF16 surrogate vs plain "
                      "exact-filter HMC (min ESS over 47 parameters)",
            "value": res["da_hmc"]["ess_per_s"], "unit": "ESS/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64 exact filter / bf16 surrogate",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "psr20_toa500-2000_w4096 TOAs with an injected model source",
                       "chains": 4096, "surrogate": "MLP 47-4x256-48 GELU, BF16, FP32 accumulate",
                       "train_rows": res["train_rows"]},
            "da_hmc": res["da_hmc"], "exact_hmc": res["hmc"], "da_clocks": leg["clocks"],
            "ess_per_s_gain": res["ess_per_s_gain"],
            "ess_per_s_gain_incl_training": res["ess_per_s_gain_incl_training"],
            "posterior_mean_z_max": res["posterior_mean_z_max"],
            "posterior_sd_ratio_range": res["posterior_sd_ratio_range"],
            "surrogate_fit": {k: res[k] for k in ("holdout_abs_err_nats_median",
                                                  "holdout_abs_err_nats_p90",
                                                  "holdout_grad_rel_err_median", "final_loss",
                                                  "data_gen_s", "train_s", "epochs")},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "k_mlp_fused (surrogate eval, 4096 rows, forward with gradient head)",
                         "kernel_ms": eval_ms, "peak_source": f"bf16_tflops ({src})",
                         "backprop_ms": bp_ms, "backprop_tflops": bp_flop / (bp_ms * 1e-3) / 1e12,
                         "train_step_ms": train_ms,
                         "train_tflops": train_flop / (train_ms * 1e-3) / 1e12},
            "clocks": clk, "experiment": res}
    print(json.dumps(line), flush=True)
    return 0


def run_surrogate(args):
    """The surrogate network's evaluation alone (random seeded weights, the
    quadratic baseline on), CUDA events over 50 calls after 5 warm-up calls.
    The sampler's mode (value + back-propagated input gradient) runs first
    with the fused kernel, so its third launch is the one to profile."""
    import numpy as np
    import torch

    from paper_2510_11077_gb300 import surrogate
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, src = _measured_peaks()
    modes = [("value backprop", 1, True), ("gradient head", 0, True), ("value", 0, False)]
    fwd_flop = 2 * (64 * 256 + 3 * 256 * 256 + 256 * 64)
    bwd_flop = 2 * (3 * 256 * 256 + 256 * 64)
    out = {}
    for rows in (4096, 16384):
        net = surrogate.Surrogate(device=local, max_rows=rows, seed=3)
        rng = np.random.default_rng(1)
        net.set_normalizers(np.zeros(47), np.ones(47), 0.0, 1.0)
        A = rng.standard_normal((47, 47)).astype(np.float32) / 47
        net.set_baseline(A @ A.T + 0.1 * np.eye(47, dtype=np.float32))
        x = torch.from_numpy(rng.standard_normal((rows, 47)).astype(np.float32)).to(dev)
        for name, gm, wg in modes:
            net.set_grad_mode(gm)
            # fused: automatic cluster size, then 1, 2 and 4 CTAs per slab; then per layer
            for fused, cl in ((True, 0), (True, 1), (True, 2), (True, 4), (False, 0)):
                net.set_fused(fused)
                net.set_cluster(cl)
                for _ in range(5):
                    net.eval(x, with_grad=wg)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(50):
                    net.eval(x, with_grad=wg)
                e1.record()
                torch.cuda.synchronize(dev)
                net.check()
                us = e0.elapsed_time(e1) / 50 * 1e3
                flop = rows * (fwd_flop + (bwd_flop if gm == 1 and wg else 0))
                tag = ("fused" + ("" if cl == 0 else f", cluster {cl}")) if fused else "per layer"
                out[f"{rows} rows, {name}, {tag}"] = {"us": us, "tflops": flop / (us * 1e-6) / 1e12}
            net.set_cluster(0)
        net.close()
    # one training step (forward with saved activations, loss, back-propagation,
    # weight gradients, Adam) on 4096-row minibatches of a resident set
    net = surrogate.Surrogate(device=local, max_rows=4096, seed=3)
    rng = np.random.default_rng(2)
    net.set_normalizers(np.zeros(47), np.ones(47), 0.0, 1.0)
    n_set = 65536
    xs = torch.from_numpy(rng.standard_normal((n_set, 47)).astype(np.float32)).to(dev)
    ls = torch.from_numpy(rng.standard_normal(n_set).astype(np.float32)).to(dev)
    gs = torch.from_numpy(rng.standard_normal((n_set, 47)).astype(np.float32)).to(dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    n_steps = n_set // 4096
    for i in range(5):
        sl = slice((i % n_steps) * 4096, (i % n_steps + 1) * 4096)
        net.train_step(xs[sl], ls[sl], gs[sl], 1e-4, loss_out=loss)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(4 * n_steps):
        sl = slice((i % n_steps) * 4096, (i % n_steps + 1) * 4096)
        net.train_step(xs[sl], ls[sl], gs[sl], 1e-4, loss_out=loss)
    e1.record()
    torch.cuda.synchronize(dev)
    net.check()
    net.close()
    us = e0.elapsed_time(e1) / (4 * n_steps) * 1e3
    # forward, the input-side gradients of layers 4..1 and every weight gradient
    train_flop = 4096 * (fwd_flop + bwd_flop + fwd_flop)
    out["4096 rows, training step"] = {"us": us, "tflops": train_flop / (us * 1e-6) / 1e12}
    key = "4096 rows, value backprop, fused"
    line = {"metric": "surrogate evaluation latency (value + back-propagated gradient, 4096 rows)",
            "value": out[key]["us"], "unit": "us", "n_gpus": 1, "higher_is_better": False,
            "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "roofline": {"bound": "tensor", "achieved": out[key]["tflops"], "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": out[key]["tflops"] / peaks["bf16_tflops"],
                         "kernel": "k_mlp_fused", "peak_source": f"bf16_tflops ({src})"},
            "runs": out}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_latency(args):
    """The latency leg alone: one parameter vector on the 1-pulsar, 1000-TOA
    array, loglik + gradient through the time-parallel filter (the line's
    value) against the sequential one, and the loglik alone."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    out = latency_leg(args, torch.device("cuda", local), local)
    g = out["gradient"]
    line = {"metric": "loglik+grad latency, one parameter vector (1 pulsar x 1000 TOAs)",
            "value": g["scan"]["median_us"], "unit": "us", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": LATENCY_WORKLOAD, "walkers": 1, "plan": "SCAN",
                       "l2": "flushed before each call"},
            "latency_1psr": out}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_gwb(args):
    """The GW-background leg alone: the joint filter's likelihood and its
    gradient for --gwb-batch parameter vectors on the 20-pulsar array."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    out = gwb_leg(args, torch.device("cuda", local), local)
    g = out["gradient"]
    line = {"metric": "joint-filter loglik+grad evals/s (Hellings-Downs GW background)",
            "value": g["value"], "unit": "evals/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": out["workload"], "batch": out["batch"],
                       "l2": "flushed before each timed call (256 MiB write, untimed)"},
            "gwb_hd": out}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "da-hmc":
        return run_da_hmc(args)
    if args.mode == "surrogate":
        return run_surrogate(args)
    if args.mode == "latency":
        return run_latency(args)
    if args.mode == "gwb":
        return run_gwb(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
