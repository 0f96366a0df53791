"""The benchmark's multi-rank aggregation (independent replicas, one map per
GPU): whole-job work is the sum over ranks, time is the slowest rank's.
Run as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = {"build_s": 1.0 + rank, "access_s": 2.0 + 3 * rank, "step_s": 3.0 + 4 * rank,
             "records": 100.0, "accesses": 10.0 * (rank + 1)}
    agg = bench.aggregate(local, world)
    out[rank] = agg
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        agg = out[r]
        assert agg["build_s"] == 2.0 and agg["access_s"] == 5.0 and agg["step_s"] == 7.0
        assert agg["records"] == 200.0 and agg["accesses"] == 30.0


def test_aggregate_single_rank_is_identity():
    import bench
    local = {"build_s": 1.5, "access_s": 2.5, "step_s": 4.0, "records": 7.0, "accesses": 9.0}
    assert bench.aggregate(local, 1) == local
