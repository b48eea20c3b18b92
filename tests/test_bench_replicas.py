"""The benchmark's multi-replica path on CPU: two ranks over gloo (one
process each, as torchrun launches them) agree on the slowest replica's time
and on the whole-job value; a single rank is unchanged."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times_ms, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks_of(times_ms[rank], world, dist, torch.device("cpu"))
        value = bench.whole_job_mlups(world, 1 << 20, 100, ms / 1e3)
        dist.barrier()
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world, port = 2, _free_port()
    times = [8.0, 9.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 9.5
    assert value == pytest.approx(2 * (1 << 20) * 100 / 9.5e-3 / 1e6)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks_of(3.25, 1, None, None) == 3.25
    assert bench.whole_job_mlups(1, 1000, 10, 0.5) == pytest.approx(0.02)
