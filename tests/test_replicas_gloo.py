"""The N>1 bench path is replicas only (the pipeline does not shard): each rank times its own
volume and the job reports the slowest rank's step with the voxels of all ranks.  This runs
that aggregation on two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    agg = bench.aggregate_replicas(10.0 * (rank + 1), 30.0 + rank, 1_000_000, dist)
    out[rank] = (agg["world"], agg["ms"], agg["e2e_ms"], agg["value"], agg["e2e_value"])
    dist.destroy_process_group()


def test_replicas_aggregate_max_time_and_all_voxels():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        world, ms, e2e_ms, value, e2e_value = res[rank]
        assert world == 2 and ms == 20.0 and e2e_ms == 31.0
        assert abs(value - 2 * 1_000_000 / 0.020 / 1e6) < 1e-9
        assert abs(e2e_value - 2 * 1_000_000 / 0.031 / 1e6) < 1e-9


def test_single_process_needs_no_process_group():
    import bench

    agg = bench.aggregate_replicas(12.5, 14.0, 2_000_000)
    assert agg["world"] == 1 and agg["ms"] == 12.5 and abs(agg["value"] - 160.0) < 1e-9
