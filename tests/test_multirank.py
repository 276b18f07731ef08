"""The multi-GPU bench path on the CPU: two gloo ranks each time their own
independent TM; the job's time is the slowest rank's and its throughput counts
every rank's rows (weak scaling, no collective on the data path)."""
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


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_seconds = 0.25 + 0.5 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(local_seconds, world, device="cpu")
        out[rank] = (t, bench.job_rows_per_s(8192, world, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_rows():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, v = res[0]
    assert t == pytest.approx(0.75)
    assert v == pytest.approx(2 * 8192 / 0.75)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.job_rows_per_s(100, 1, 0.5) == 200.0
