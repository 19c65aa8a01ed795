"""Host side of the y-slab decomposition of one run (tfkt_slab_* in include/tfkt.h).

A run of ny rows is split into contiguous slabs of owned rows; each slab context
also holds GHOST rows on each side, which must be replaced with the neighbours'
current rows before every step (one step of the scheme of Sec. VI reads data at
most three rows away; the width is a whole tile row so that the slabs keep the
single-domain run's tiles). This module holds what needs no GPU: the partition of
the rows, the global rows of a slab's local rows, the perturbation of those rows,
and the exchange itself, written against pack/unpack callables so that it drives
slab contexts in one process (device buffers) or across torch.distributed ranks
(host buffers) alike.

Message routing: a slab's HIGH side (larger y) goes to the next slab's LOW ghost
rows, its LOW side to the previous slab's HIGH ghost rows; the slabs form a ring
(the run is periodic in y).
"""
from __future__ import annotations

import numpy as np

GHOST = 8          # TFKT_SLAB_GHOST: one row of 32 x 8 tiles
LOW, HIGH = 0, 1   # TFKT_SLAB_LOW, TFKT_SLAB_HIGH
TAG_UP, TAG_DOWN = 11, 12   # a HIGH pack travels up to a LOW unpack; a LOW pack down


def partition(ny: int, parts: int, align: int = 8) -> list[tuple[int, int]]:
    """(y0, rows) of `parts` contiguous slabs covering [0, ny): sizes differ by at
    most `align` rows and are multiples of `align` when ny is (so that every slab
    keeps the fused path), and every slab holds at least GHOST rows."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    unit = align if ny % align == 0 else 1
    units = ny // unit
    if units < parts or (ny // parts) < GHOST:
        raise ValueError(f"{ny} rows cannot make {parts} slabs of at least {GHOST} rows")
    base, extra = divmod(units, parts)
    out, y0 = [], 0
    for k in range(parts):
        n = (base + (1 if k < extra else 0)) * unit
        out.append((y0, n))
        y0 += n
    assert y0 == ny
    return out


def neighbours(k: int, parts: int) -> tuple[int, int]:
    """(slab below, slab above) of slab k on the periodic ring."""
    return (k - 1) % parts, (k + 1) % parts


def extended_rows(y0: int, n: int, ny: int, ghost: int = GHOST) -> np.ndarray:
    """Global rows of a slab's local rows: y0 - ghost ... y0 + n + ghost - 1 (mod ny)."""
    return np.arange(y0 - ghost, y0 + n + ghost) % ny


def local_perturbation(pert: np.ndarray, y0: int, n: int, ghost: int = GHOST) -> np.ndarray:
    """The whole run's perturbation [2, ny, nx] at a slab's local rows."""
    return np.ascontiguousarray(pert[:, extended_rows(y0, n, pert.shape[1], ghost), :])


def exchange_local(slabs, bufs, sync=None):
    """Refresh the ghost rows of slabs held by one process. slabs[k] has
    pack(side, ptr, nbytes, device) / unpack(...) / halo_bytes(); bufs[k] is a pair
    of device buffers (objects with data_ptr()) for its LOW and HIGH packs. Every
    pack is taken before any unpack (the two touch disjoint rows, but a slab's
    neighbour may be itself); the copies run on the slabs' streams, which `sync`
    (if given) must order between the packs and the unpacks."""
    parts = len(slabs)
    nb = [s.halo_bytes() for s in slabs]
    for k, s in enumerate(slabs):
        s.pack(LOW, bufs[k][LOW].data_ptr(), nb[k], True)
        s.pack(HIGH, bufs[k][HIGH].data_ptr(), nb[k], True)
    if sync is not None:
        sync()
    for k, s in enumerate(slabs):
        lo, hi = neighbours(k, parts)
        s.unpack(LOW, bufs[lo][HIGH].data_ptr(), nb[k], True)
        s.unpack(HIGH, bufs[hi][LOW].data_ptr(), nb[k], True)


def exchange_ranks(pack, unpack, send, recv, dist, rank: int, world: int):
    """Refresh one rank's ghost rows from its neighbours' owned rows over a
    torch.distributed process group with host (CPU) buffers. pack(side, tensor)
    fills tensor with that side's rows, unpack(side, tensor) writes them into the
    ghost rows; send and recv are pairs (LOW, HIGH) of uint8 CPU tensors of the
    message size. With one rank the slab is its own neighbour on both sides."""
    pack(LOW, send[LOW])
    pack(HIGH, send[HIGH])
    if world == 1:
        unpack(LOW, send[HIGH])
        unpack(HIGH, send[LOW])
        return
    lo, hi = neighbours(rank, world)
    reqs = [dist.isend(send[HIGH], dst=hi, tag=TAG_UP),
            dist.isend(send[LOW], dst=lo, tag=TAG_DOWN),
            dist.irecv(recv[LOW], src=lo, tag=TAG_UP),
            dist.irecv(recv[HIGH], src=hi, tag=TAG_DOWN)]
    for r in reqs:
        r.wait()
    unpack(LOW, recv[LOW])
    unpack(HIGH, recv[HIGH])
