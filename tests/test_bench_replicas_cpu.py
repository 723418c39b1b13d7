"""Multi-process host logic of bench.py (replicas: one registration per rank,
max-over-ranks timing, whole-job aggregate), on CPU with the gloo backend and
two ranks."""
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


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        mx = bench.max_over_ranks(times[rank], dist, "cpu")
        rate = bench.whole_job_rate(1000.0, 4, world, mx)
        out[rank] = (mx, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate():
    world, port = 2, _free_port()
    times = [120.0, 180.0]  # ms of each rank's timed region
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        got = dict(out)
    for r in range(world):
        mx, rate = got[r]
        assert mx == 180.0                        # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 * 4 / 0.180)  # all ranks' units / that time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.whole_job_rate(10.0, 3, 1, 1000.0) == pytest.approx(30.0)
