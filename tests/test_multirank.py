"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each
timing its own replica's batch; every rank agrees on the slowest rank's time
and the whole-job rate counts the queries of all ranks (weak scaling, no
data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, _ = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        mine = 1.0 + r  # rank 1 is the slower one
        t = bench.max_over_ranks(mine, dist, "cpu")
        out[r] = (t, bench.job_rate(w, 5, 1000, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        got = dict(out)
    assert set(got) == {0, 1}
    for r in range(world):
        t, rate = got[r]
        assert t == 2.0
        assert rate == world * 5 * 1000 / 2.0


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_rate(1, 4, 10, 2.0) == 20.0
