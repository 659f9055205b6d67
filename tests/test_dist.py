"""The multi-GPU path of bench.py is replicas only: each rank gauge-fixes its
own copy and the job reports the sum of the ranks' site updates over the
slowest rank's time. The aggregation is checked here with gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate(10.0 * (rank + 1), 1000 * (rank + 1), world)
    out[rank] = (ms, units)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation_with_gloo(world):
    ctx = torch.multiprocessing.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    expect_ms = 10.0 * world
    expect_units = 1000 * world * (world + 1) / 2
    for r in range(world):
        assert out[r] == (expect_ms, expect_units)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(3.5, 42, 1) == (3.5, 42)
