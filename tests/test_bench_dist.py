"""Multi-replica aggregation of bench.py on CPU with gloo, world size 2: the job's
throughput is every rank's site updates over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [100.0, 250.0][rank]
    mlups, ms_max = bench.aggregate_mlups(1e6 * 50, world, ms_local, device="cpu")
    out[rank] = (mlups, ms_max)
    dist.destroy_process_group()


def test_two_rank_aggregation():
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
        mlups, ms_max = out[r]
        assert ms_max == 250.0
        assert mlups == pytest.approx(2 * 1e6 * 50 / 0.25 / 1e6)
