"""Host side of the y-slab decomposition, without a GPU: the partition of
the rows, the local rows a slab holds, the halo schedule between ranks
(world_size 2 and 3, gloo, walls and periodic y) and the combination of the
slabs' diagnostics."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _slabs():
    from paper_2111_00847_gb300 import slabs

    return slabs


def test_partition_covers_the_rows():
    slabs = _slabs()
    for ny, parts in ((150, 2), (150, 3), (16384 * 4, 4), (33, 8)):
        bands = slabs.partition(ny, parts)
        assert len(bands) == parts
        assert bands[0][0] == 0
        for (a, ha), (b, _) in zip(bands, bands[1:]):
            assert a + ha == b
        assert bands[-1][0] + bands[-1][1] == ny
        assert max(h for _, h in bands) - min(h for _, h in bands) <= 1
    with pytest.raises(ValueError):
        slabs.partition(10, 3)  # fewer than LBM_SLAB_GHOST rows a slab


def test_neighbours_and_local_rows():
    slabs = _slabs()
    assert slabs.neighbours(0, 3, False) == (None, 1)
    assert slabs.neighbours(2, 3, False) == (1, None)
    assert slabs.neighbours(0, 3, True) == (2, 1)
    assert slabs.neighbours(1, 2, True) == (0, 0)
    # a middle slab of a walled grid, and the first slab of a periodic one
    assert list(slabs.local_rows(20, 8, 6, 4, 4)) == list(range(4, 18))
    assert list(slabs.local_rows(20, 0, 6, 4, 4)) == [16, 17, 18, 19, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, periodic, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slabs = _slabs()
    n = 16
    # each message carries its origin: rank * 10 + (1: bottom, 2: top)
    send_lo = torch.full((n,), rank * 10 + 1, dtype=torch.uint8)
    send_hi = torch.full((n,), rank * 10 + 2, dtype=torch.uint8)
    recv_lo = torch.zeros(n, dtype=torch.uint8)
    recv_hi = torch.zeros(n, dtype=torch.uint8)
    for _ in range(3):  # repeated exchanges stay matched
        slabs.exchange_messages(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic, dist)
    q.put((rank, int(recv_lo.min()), int(recv_lo.max()), int(recv_hi.min()), int(recv_hi.max())))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("periodic", [False, True], ids=["walls", "periodic"])
def test_halo_schedule_gloo(world, periodic):
    """Each rank's bottom ghost rows receive its lower neighbour's top
    message and its top ghost rows its upper neighbour's bottom message;
    sides at a global wall receive nothing."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(world, periodic, _free_port(), q), nprocs=world, start_method="spawn")
    got = sorted(q.get() for _ in range(world))
    slabs = _slabs()
    for rank, lo_min, lo_max, hi_min, hi_max in got:
        lower, upper = slabs.neighbours(rank, world, periodic)
        assert lo_min == lo_max and hi_min == hi_max
        assert lo_min == (0 if lower is None else lower * 10 + 2)
        assert hi_min == (0 if upper is None else upper * 10 + 1)


def test_combine_diag():
    slabs = _slabs()
    a = dict(t=5, sum_phi=10.0, Du_rms=2.0, Sm_rms=1.0, umax=0.1, nonfinite=0.0, n_avg=100.0, reserved=0.0)
    b = dict(t=5, sum_phi=5.0, Du_rms=1.0, Sm_rms=3.0, umax=0.3, nonfinite=1.0, n_avg=300.0, reserved=0.0)
    d = slabs.combine_diag([a, b])
    assert d["sum_phi"] == 15.0 and d["umax"] == 0.3 and d["nonfinite"] == 1.0 and d["n_avg"] == 400.0
    assert d["Du_rms"] == pytest.approx(np.sqrt((4 * 100 + 1 * 300) / 400))
    assert d["Sm_rms"] == pytest.approx(np.sqrt((1 * 100 + 9 * 300) / 400))
