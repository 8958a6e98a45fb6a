"""The multi-rank path of bench.py (replicas only: every rank runs its own
copy of the workload, no collective on the data path): the step time is the
maximum over ranks and the throughput counts every rank's units.  Two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + rank, 3.0 - rank]          # rank-dependent step and e2e times (ms)
    got = bench.max_over_ranks(local, torch.device("cpu"))
    value = bench.replica_throughput(world, 1000.0, got[0])
    out.put((rank, got, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_the_units():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [11.0, 3.0]                      # max over ranks, element-wise
        assert value == pytest.approx(2 * 1000.0 / 11.0e-3)


def test_single_process_keeps_its_values():
    import torch
    import bench
    assert bench.max_over_ranks([1.5, 2.5], torch.device("cpu")) == [1.5, 2.5]
