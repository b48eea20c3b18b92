"""y-slab decomposition of one grid: partition, halo schedule and exchange.

A grid of ny rows is divided into bands of rows, one ``Simulation`` (a
y-slab handle, ``lbm_create_slab``) per band.  After every step each slab
sends the ``LBM_SLAB_GHOST`` own rows next to a side that borders another
slab (f and g, post-collision, one message per side) and writes the message
it receives into its ghost rows (``lbm_slab_pack`` / ``lbm_slab_unpack``).
The library does the packing on the device; this module only orders the
copies: device-to-device for slabs in one process, ``torch.distributed``
point-to-point (NCCL between GPUs, gloo on the host) across processes.
"""
from __future__ import annotations

import numpy as np

from . import LBM_BOTTOM, LBM_SLAB_GHOST, LBM_TOP, Simulation

# tags of the two message directions (gloo matches on them; NCCL matches the
# point-to-point operations between a pair in the order they are posted,
# which the fixed order in exchange_messages keeps consistent on both ends)
TAG_DOWN, TAG_UP = 11, 12


def partition(ny: int, parts: int) -> list[tuple[int, int]]:
    """Bands (y_lo, ny_own) of near-equal height covering [0, ny)."""
    if parts < 2 or ny < parts * LBM_SLAB_GHOST:
        raise ValueError(f"{ny} rows do not split into {parts} slabs of at least {LBM_SLAB_GHOST} rows")
    base, extra = divmod(ny, parts)
    out, y = [], 0
    for k in range(parts):
        h = base + (1 if k < extra else 0)
        out.append((y, h))
        y += h
    return out


def neighbours(rank: int, world: int, periodic: bool) -> tuple[int | None, int | None]:
    """(lower, upper) neighbour ranks of a slab; None beyond a global wall."""
    lower = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    upper = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return lower, upper


def local_rows(ny: int, y_lo: int, ny_own: int, ghost_lo: int, ghost_hi: int) -> np.ndarray:
    """Global row index of every local row of a slab (wrapped: with walls the
    ghost rows never leave [0, ny))."""
    return np.arange(y_lo - ghost_lo, y_lo + ny_own + ghost_hi) % ny


def local_field(field: np.ndarray | None, sim: Simulation) -> np.ndarray | None:
    """The rows of a global [ny][nx] field that a slab's local grid holds."""
    if field is None:
        return None
    y_lo, own, glo, ghi = sim.slab
    return np.ascontiguousarray(field[local_rows(field.shape[0], y_lo, own, glo, ghi)])


def exchange_messages(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, periodic: bool, dist,
                      group=None):
    """Point-to-point transport of one halo exchange.  send_lo / send_hi: this
    rank's bottom / top messages; recv_lo / recv_hi: buffers for the messages
    of the lower / upper neighbour (received into this rank's bottom / top
    ghost rows).  Buffers of a side without a neighbour may be None."""
    lower, upper = neighbours(rank, world, periodic)
    ops = []
    if lower is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lower, group, TAG_DOWN))
    if upper is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, upper, group, TAG_UP))
    if upper is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, upper, group, TAG_DOWN))
    if lower is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lower, group, TAG_UP))
    # one batch: every send and receive of the exchange is posted together
    # (NCCL group semantics), so no ordering of the pairs can deadlock
    for req in dist.batch_isend_irecv(ops) if ops else []:
        req.wait()


class HaloBuffers:
    """Device buffers of one slab's four messages (torch uint8 tensors)."""

    def __init__(self, sim: Simulation):
        import torch

        n = sim.halo_bytes
        dev = torch.device("cuda", torch.cuda.current_device())
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = (
            torch.empty(n, dtype=torch.uint8, device=dev) for _ in range(4))


def exchange_dist(sim: Simulation, bufs: HaloBuffers, rank: int, world: int, periodic: bool, dist, group=None):
    """One halo exchange of this rank's slab with its neighbours' processes."""
    lower, upper = neighbours(rank, world, periodic)
    if lower is not None:
        sim.pack(LBM_BOTTOM, bufs.send_lo)
    if upper is not None:
        sim.pack(LBM_TOP, bufs.send_hi)
    exchange_messages(bufs.send_lo, bufs.send_hi, bufs.recv_lo, bufs.recv_hi, rank, world, periodic, dist, group)
    if lower is not None:
        sim.unpack(LBM_BOTTOM, bufs.recv_lo)
    if upper is not None:
        sim.unpack(LBM_TOP, bufs.recv_hi)


def exchange_local(sims: list[Simulation], periodic: bool, bufs: list[HaloBuffers] | None = None):
    """One halo exchange among slabs held in this process (in band order),
    by device-to-device copies on the slabs' streams."""
    world = len(sims)
    bufs = bufs or [HaloBuffers(s) for s in sims]
    for k, s in enumerate(sims):
        lower, upper = neighbours(k, world, periodic)
        if lower is not None:
            s.pack(LBM_BOTTOM, bufs[k].send_lo)
        if upper is not None:
            s.pack(LBM_TOP, bufs[k].send_hi)
    _sync(sims)
    for k, s in enumerate(sims):
        lower, upper = neighbours(k, world, periodic)
        if lower is not None:
            s.unpack(LBM_BOTTOM, bufs[lower].send_hi)
        if upper is not None:
            s.unpack(LBM_TOP, bufs[upper].send_lo)
    _sync(sims)
    return bufs


def _sync(sims):
    streams = {id(s.stream_obj): s.stream_obj for s in sims if hasattr(s.stream_obj, "synchronize")}
    if len(streams) > 1:
        for st in streams.values():
            st.synchronize()


def combine_diag(diags: list[dict]) -> dict:
    """Diagnostics of the undivided grid from its slabs' records: sums add,
    rms values combine weighted by their node counts, max|u| is the max."""
    n = sum(d["n_avg"] for d in diags)
    out = dict(diags[0])
    out["sum_phi"] = sum(d["sum_phi"] for d in diags)
    out["nonfinite"] = sum(d["nonfinite"] for d in diags)
    out["umax"] = max(d["umax"] for d in diags)
    out["n_avg"] = n
    for k in ("Du_rms", "Sm_rms"):
        out[k] = float(np.sqrt(sum(d[k] ** 2 * d["n_avg"] for d in diags) / n)) if n else 0.0
    return out
