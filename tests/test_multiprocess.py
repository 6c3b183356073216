"""The N > 1 path of bench.py on CPU (gloo, world size 2).  Single-matrix
workloads run independent replicas joined only by the max-over-ranks step
time; the ragged batch is split across ranks in shares of nearly equal sum
n^3, each rank solving its share with no exchange, and the whole-job value is
the instances of all ranks over the slowest rank's time.  The hot path itself
has no exchange step, so these reductions are the only collectives."""
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


def _ragged_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as wl
    ns = [int(n) for n in wl.ragged_sizes(512, 0)]
    mine = bench.partition_by_work(ns, world)[rank]
    # every rank's share, gathered to check the split
    share = torch.zeros(512, dtype=torch.int64)
    share[mine] = rank + 1
    dist.all_reduce(share)
    work = torch.tensor([float(sum(ns[b] ** 3 for b in mine))], dtype=torch.float64)
    works = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(works, work)
    # whole-job value: instances of all ranks over the slowest rank's time
    t_local = 0.030 if rank == 0 else 0.040
    value, tmax = bench.aggregate(t_local, world, float(len(mine)))
    q.put((rank, share.tolist(), [float(w) for w in works], value, tmax, len(mine)))
    dist.barrier()
    dist.destroy_process_group()


def test_ragged_batch_split_by_sum_n3_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ragged_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    counts = {r: c for r, _, _, _, _, c in out}
    for rank, share, works, value, tmax, _ in out:
        # every instance in exactly one share (the all-reduced labels are 1 or 2)
        assert sorted(set(share)) == [1, 2]
        assert share.count(1) == counts[0] and share.count(2) == counts[1]
        # the shares' sum n^3 agree to within the largest single instance
        assert abs(works[0] - works[1]) <= 768 ** 3
        assert tmax == pytest.approx(0.040)
        assert value == pytest.approx(512 / 0.040)


def test_partition_covers_and_balances():
    import bench
    ns = [5, 3, 3, 2, 2, 2, 1]
    parts = bench.partition_by_work(ns, 3)
    assert sorted(b for p in parts for b in p) == list(range(len(ns)))
    loads = [sum(ns[b] ** 3 for b in p) for p in parts]
    assert sorted(loads) == [36, 43, 125]          # largest first, each to the lightest share
    assert bench.partition_by_work(ns, 1) == [list(range(len(ns)))]
