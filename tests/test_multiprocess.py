"""The N > 1 path of bench.py on CPU: independent replicas joined only by the
max-over-ranks step time (gloo, world size 2).  The hot path itself has no
exchange step, so this is the only collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 0.010 if rank == 0 else 0.025
    value, tmax = bench.aggregate(t_local, world)
    q.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, value, tmax in out:
        assert tmax == pytest.approx(0.025)
        assert value == pytest.approx(2 / 0.025)


def test_single_rank_aggregation():
    import bench
    v, t = bench.aggregate(0.02, 1)
    assert v == pytest.approx(50.0) and t == pytest.approx(0.02)
