"""The N > 1 path of bench.py on CPU: independent replicas, one per rank, with
the job's time the slowest rank's (max over ranks through a collective) and
the value the units of all ranks over that time.  Two gloo ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = bench.max_over_ranks(dist, 1.0 + rank, device="cpu")
        value = bench.replicas_value(world, 1000, 5, secs)
        q.put((rank, secs, value))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_units():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, secs, value in got:
        assert secs == pytest.approx(2.0)
        assert value == pytest.approx(2 * 1000 * 5 / 2.0)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.replicas_value(1, 10, 4, 2.0) == 20.0
