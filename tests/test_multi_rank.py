"""The multi-GPU path runs independent replicas: the only cross-rank
traffic is the timing aggregation (max of the timed spans, sum of the units
processed).  Checked here with world_size 2 over gloo on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "timed" (10 + 5 r) ms and processed (8 + r) requests
    ms, units = bench.aggregate(10.0 + 5 * rank, 8 + rank, dist, "cpu")
    dist.barrier()
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_replica_timing_aggregation_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest span and the total work
    assert all(ms == 15.0 and units == 17 for _, ms, units in res)


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 8) == (12.5, 8)
