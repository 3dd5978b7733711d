"""The multi-rank bookkeeping of bench.py (replicas, max over ranks) on two
gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    m = bench.max_over_ranks(100.0 + 10.0 * rank, world)
    v = bench.aggregate_seconds(m, world)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        m, v = out[r]
        assert m == 110.0            # the slowest rank sets the step time
        assert abs(v - 0.055) < 1e-12   # two solves per 110 ms step
