"""Multi-process host logic on the CPU (gloo, world size 2): the portfolio
partition every rank computes locally, the max-over-ranks job time and the
whole-job rate of bench.py.  No GPU."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_15629_b300 import dist as D


def test_lpt_partition_is_a_balanced_partition():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0.0, 1.0, size=256)
    for world in (1, 2, 3, 8):
        parts = D.shard_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))          # every unit once
        loads = [costs[p].sum() for p in parts]
        # LPT: the most loaded rank exceeds the mean by at most one unit
        assert max(loads) <= costs.sum() / world + costs.max() + 1e-9
    assert D.shard_by_cost([5.0, 1.0, 1.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3, 4, 5]]
    with pytest.raises(ValueError):
        D.shard_by_cost([1.0], 0)


def test_rate_is_whole_job():
    assert D.aggregate_rate(100.0, 4, 2.0) == 200.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, costs):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = D.shard_by_cost(costs, world)[rank]
        # a rank's "time" is its load; the job time is the slowest rank's
        local = float(np.asarray(costs)[mine].sum())
        job = D.job_seconds(local, torch)
        rate = D.aggregate_rate(len(costs) / world, world, job)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{','.join(map(str, mine))};{local!r};{job!r};{rate!r}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_max_time():
    costs = [float(c) for c in np.random.default_rng(1).uniform(1.0, 10.0, size=37)]
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(2, _free_port(), d, costs), nprocs=2, join=True)
        rows = [open(os.path.join(d, f"r{r}.txt")).read().split(";") for r in range(2)]
    mine = [[int(x) for x in r[0].split(",") if x] for r in rows]
    local = [float(r[1]) for r in rows]
    job = [float(r[2]) for r in rows]
    assert sorted(mine[0] + mine[1]) == list(range(len(costs)))   # no unit lost or doubled
    assert not set(mine[0]) & set(mine[1])
    assert job[0] == job[1] == max(local)                          # max over ranks, agreed
    assert float(rows[0][3]) == pytest.approx(len(costs) / max(local))
