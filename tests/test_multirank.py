"""The multi-process path of bench.py on CPU: two gloo ranks (one process each), as torchrun would
start them, reduce their timings to the slowest rank and report the whole-job rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.reduce_max(0.5 + rank, world, "cpu")  # rank r took 0.5 + r seconds
        rate = bench.whole_job_rate(100.0, t, world)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_slowest():
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the job moved 2 x 100 units in 1.5 s
    assert [t for _, t, _ in res] == [1.5, 1.5]
    assert all(abs(rate - 200.0 / 1.5) < 1e-9 for _, _, rate in res)


def test_one_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(0.25, 1) == 0.25
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0
