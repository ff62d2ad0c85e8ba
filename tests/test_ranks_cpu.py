"""Multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each a replica
of the workload, must agree on the step count, take the slowest rank's time
and report the units of all ranks (weak scaling).  No GPU involved."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 1 is slower; both processed the same units per step
        total_ms = 100.0 if rank == 0 else 160.0
        out = bench.aggregate_ranks(total_ms=total_ms, units_per_step=1000, steps=4, world=world, device=None)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        total_ms, value = got[rank]
        assert total_ms == pytest.approx(160.0)
        # 1000 units x 4 steps x 2 ranks over the slowest rank's 0.16 s
        assert value == pytest.approx(1000 * 4 * 2 / 0.160)


def test_single_rank_needs_no_process_group():
    total_ms, value = bench.aggregate_ranks(total_ms=50.0, units_per_step=10, steps=5, world=1, device=None)
    assert total_ms == 50.0 and value == pytest.approx(10 * 5 / 0.05)
