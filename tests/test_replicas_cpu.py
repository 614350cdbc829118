"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas) agree on the
slowest rank's time, and the whole-job rate counts every rank's cells over
that time.  No GPU is involved."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total = 2.0 + 3.0 * rank                       # rank 1 is the slow one
        slow = bench.slowest_rank_time(total, world, "cpu")
        rate = bench.whole_job_rate(1e9, world, slow, 10)
        q.put((rank, slow, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [5.0, 5.0]                  # both ranks see the slowest time
    assert out[0][2] == pytest.approx(2 * 1e9 / (5.0 / 10))   # all ranks' units over it


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_time(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(4e10, 1, 3.5, 10) == pytest.approx(4e10 / 0.35)
