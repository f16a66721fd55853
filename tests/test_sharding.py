"""Sharding of batched solves over ranks: the plan, and the gather over real
gloo ranks on the CPU (the GPU solve is replaced by a stand-in that reports
which systems it was given)."""
import os
import socket

import pytest

from paper_1808_05506_gb300 import sharding


def test_assignment_covers_each_system_once_and_balances():
    import numpy as np
    rng = np.random.default_rng(3)
    nvs = [int(v) for v in rng.integers(1, 25, 48)]
    for world in (1, 2, 3, 4, 8):
        plan = sharding.assign_systems(nvs, world)
        flat = sorted(i for p in plan for i in p)
        assert flat == list(range(48))
        loads = [sum(nvs[i] for i in p) for p in plan]
        # greedy largest-first: the spread is at most the largest single system
        assert max(loads) - min(loads) <= max(nvs)
        assert plan == sharding.assign_systems(nvs, world)   # deterministic


def test_assignment_more_ranks_than_systems():
    plan = sharding.assign_systems([5, 1], 4)
    assert sorted(i for p in plan for i in p) == [0, 1]
    assert sum(1 for p in plan if not p) == 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nvs, out_dir):
    import json
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def fake_solve(bs, masses, **kw):
        stats = [{"converged": 1, "outer_iterations": 2, "residual_max": 1e-11 * b} for b in bs]
        return [None] * len(bs), None, stats, {}, 0

    local, xs, status, stats, totals = sharding.solve_batched_sharded(
        fake_solve, nvs, [0.12] * len(nvs), lambda i: i, rank, world, tol=1e-10)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"local": local, "stats": stats}, f)
    dist.destroy_process_group()


def test_sharded_solve_gathers_every_system_once(tmp_path):
    import json
    import torch.multiprocessing as mp
    nvs = [7, 3, 12, 1, 24, 5, 9]
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), nvs, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    plan = sharding.assign_systems(nvs, world)
    for r in range(world):
        assert res[r]["local"] == plan[r]
        # every rank sees the statistics of all systems, in system order, each once
        assert [s["system"] for s in res[r]["stats"]] == list(range(len(nvs)))
        for s in res[r]["stats"]:
            assert s["rank"] in (0, 1) and s["system"] in plan[s["rank"]]
            assert s["residual_max"] == pytest.approx(1e-11 * s["system"])
