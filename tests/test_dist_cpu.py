"""The multi-rank path on CPU: two gloo ranks shard walkers with no data-path
collective, and the job time is the maximum over ranks."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import kalman
    from paper_2510_11077_gb300 import dist as pdist, inputs
    data = inputs.make_array(np.array([60, 25]), seed=5)
    theta = inputs.make_theta_batch(data, 4, seed=pdist.rank_seed(100, rank))
    ll = kalman.loglik(data, theta)
    fake_seconds = 1.0 + rank                     # rank 1 is the slow one
    tmax = pdist.max_over_ranks(fake_seconds)
    value = pdist.job_throughput(len(theta), world, tmax)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, theta, ll))
    if rank == 0:
        np.save(os.path.join(out_dir, "result.npy"),
                np.array([tmax, value], dtype=np.float64))
        for r, th, l in gathered:
            np.save(os.path.join(out_dir, f"theta{r}.npy"), th)
            np.save(os.path.join(out_dir, f"ll{r}.npy"), l)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_walkers(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    tmax, value = np.load(tmp_path / "result.npy")
    assert tmax == 2.0 and value == pytest.approx(2 * 4 / 2.0)
    th0, th1 = np.load(tmp_path / "theta0.npy"), np.load(tmp_path / "theta1.npy")
    assert not np.any(np.all(th0[:, None, :] == th1[None, :, :], axis=2))   # disjoint shards
    # each rank's results equal a single-process evaluation of its shard
    from oracle import kalman
    from paper_2510_11077_gb300 import inputs
    data = inputs.make_array(np.array([60, 25]), seed=5)
    for r in (0, 1):
        th = np.load(tmp_path / f"theta{r}.npy")
        assert np.array_equal(np.load(tmp_path / f"ll{r}.npy"), kalman.loglik(data, th))


def _timed_worker(rank, world, port, out_dir):
    """The bench's timing protocol on gloo ranks: each rank times its own
    oracle steps (rank 1 deliberately slower), and the job time is the
    maximum over ranks of each rank's total."""
    import time

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import kalman
    from paper_2510_11077_gb300 import dist as pdist, inputs
    w, r, lr = pdist.env()
    data = inputs.make_array(np.array([40, 30]), seed=8)
    theta = inputs.make_theta_batch(data, 3, seed=pdist.rank_seed(200, r))
    calls = {"warm": 0, "timed": 0, "started": None}

    def step(timed):
        t0 = time.perf_counter()
        kalman.loglik(data, theta)
        time.sleep(0.05 * (1 + r))               # rank 1 takes twice as long
        if not timed:
            calls["warm"] += 1
            return None
        calls["timed"] += 1
        return time.perf_counter() - t0

    secs, tmax = pdist.timed_steps(step, 4, 3, on_start=lambda: calls.update(started=calls["timed"]))
    value = pdist.job_throughput(len(theta) * 4, w, tmax)
    gathered = [None] * w
    dist.all_gather_object(gathered, (r, lr, w, sum(secs), tmax, value, calls))
    if r == 0:
        import json
        with open(os.path.join(out_dir, "timed.json"), "w") as f:
            json.dump(gathered, f)
    pdist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_like_the_bench(tmp_path):
    import json
    port = _free_port()
    mp.start_processes(_timed_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    rows = json.load(open(tmp_path / "timed.json"))
    assert [r[0] for r in rows] == [0, 1] and [r[1] for r in rows] == [0, 1]
    totals = [r[3] for r in rows]
    for rk, lr, w, total, tmax, value, calls in rows:
        assert w == 2 and calls == {"warm": 3, "timed": 4, "started": 0}
        assert tmax == max(totals)                      # every rank sees the job time
        assert value == 2 * 3 * 4 / tmax                # all ranks' walkers over it
    assert totals[1] > totals[0] and totals[1] >= 4 * 0.1


def test_single_process_helpers():
    from paper_2510_11077_gb300 import dist as pdist
    assert pdist.max_over_ranks(3.5) == 3.5
    assert pdist.rank_seed(10, 0) == 10 and pdist.rank_seed(10, 1) != 10
    assert pdist.job_throughput(16384, 4, 2.0) == 16384 * 2
    assert pdist.env() == (1, 0, 0) or "WORLD_SIZE" in os.environ
    secs, tmax = pdist.timed_steps(lambda timed: 0.25 if timed else None, 3, 2)
    assert secs == [0.25] * 3 and tmax == 0.75
