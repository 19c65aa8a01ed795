"""Host logic of the y-slab decomposition (paper_2201_10132_gb300/slabs.py): the
row partition, the global rows of a slab's local rows, and the ghost-row
exchange protocol, here on fake slabs (numpy rows of a seeded global array)
over world-size 2 and 3 gloo process groups on the CPU and in one process."""
import os
import socket

import numpy as np
import pytest

from paper_2201_10132_gb300 import slabs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ghost_width_matches_the_header():
    text = open(os.path.join(ROOT, "include", "tfkt.h")).read()
    assert f"#define TFKT_SLAB_GHOST {S.GHOST}" in text
    assert "TFKT_SLAB_LOW = 0, TFKT_SLAB_HIGH = 1" in text and (S.LOW, S.HIGH) == (0, 1)


@pytest.mark.parametrize("ny,parts", [(64, 2), (64, 3), (48, 5), (70, 3), (4096, 8), (40, 1)])
def test_partition_covers_the_rows(ny, parts):
    p = S.partition(ny, parts)
    assert len(p) == parts and p[0][0] == 0
    assert all(p[k][0] + p[k][1] == p[k + 1][0] for k in range(parts - 1))
    assert p[-1][0] + p[-1][1] == ny
    sizes = [n for _, n in p]
    assert min(sizes) >= S.GHOST and max(sizes) - min(sizes) <= 8
    if ny % 8 == 0:
        assert all(n % 8 == 0 for n in sizes)


def test_partition_rejects_too_many_slabs():
    with pytest.raises(ValueError):
        S.partition(32, 5)
    with pytest.raises(ValueError):
        S.partition(16, 0)


def test_extended_rows_and_local_perturbation():
    ny, nx, g = 40, 3, S.GHOST
    assert S.extended_rows(0, 16, ny).tolist() == list(range(ny - g, ny)) + list(range(16 + g))
    assert S.extended_rows(24, 16, ny).tolist() == list(range(24 - g, ny)) + list(range(g))
    pert = np.random.default_rng(0).standard_normal((2, ny, nx))
    loc = S.local_perturbation(pert, 24, 16)
    assert loc.shape == (2, 16 + 2 * g, nx) and loc.flags.c_contiguous
    assert np.array_equal(loc[:, g], pert[:, 24]) and np.array_equal(loc[:, -1], pert[:, g - 1])


class FakeSlab:
    """Owned rows of a global array plus ghost rows filled with garbage."""

    def __init__(self, glob, y0, n):
        self.glob_rows = S.extended_rows(y0, n, glob.shape[0])
        self.a = glob[self.glob_rows].copy()
        self.a[:S.GHOST] = -1.0
        self.a[-S.GHOST:] = -2.0
        self.n = n

    def rows(self, side, ghost):
        g = S.GHOST
        if ghost:
            return slice(0, g) if side == S.LOW else slice(self.n + g, self.n + 2 * g)
        return slice(g, 2 * g) if side == S.LOW else slice(self.n, self.n + g)


def _fake_run(rank, world, port, ny, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    glob = np.random.default_rng(5).standard_normal((ny, 6))
    y0, n = S.partition(ny, world)[rank]
    s = FakeSlab(glob, y0, n)
    nbytes = S.GHOST * 6 * 8
    send = [torch.zeros(nbytes, dtype=torch.uint8) for _ in range(2)]
    recv = [torch.zeros(nbytes, dtype=torch.uint8) for _ in range(2)]

    def pack(side, t):
        t.numpy()[:] = np.ascontiguousarray(s.a[s.rows(side, False)]).view(np.uint8).ravel()

    def unpack(side, t):
        s.a[s.rows(side, True)] = t.numpy().view(np.float64).reshape(S.GHOST, 6)

    S.exchange_ranks(pack, unpack, send, recv, dist, rank, world)
    ok = np.array_equal(s.a, glob[s.glob_rows])
    dist.barrier()
    dist.destroy_process_group()
    with open(f"{out}.{rank}", "w") as f:
        f.write("ok" if ok else "bad")


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_over_gloo_ranks(tmp_path, world):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res")
    mp.spawn(_fake_run, args=(world, _free_port(), 48, out), nprocs=world, join=True)
    for r in range(world):
        assert open(f"{out}.{r}").read() == "ok", r


def test_exchange_in_one_rank():
    class Dist:
        pass
    glob = np.random.default_rng(6).standard_normal((24, 4))
    s = FakeSlab(glob, 0, 24)
    import torch
    send = [torch.zeros(S.GHOST * 4 * 8, dtype=torch.uint8) for _ in range(2)]

    def pack(side, t):
        t.numpy()[:] = np.ascontiguousarray(s.a[s.rows(side, False)]).view(np.uint8).ravel()

    def unpack(side, t):
        s.a[s.rows(side, True)] = t.numpy().view(np.float64).reshape(S.GHOST, 4)

    S.exchange_ranks(pack, unpack, send, None, Dist(), 0, 1)
    assert np.array_equal(s.a, glob[s.glob_rows])


def test_exchange_local_routes_packs_to_neighbours():
    glob = np.random.default_rng(7).standard_normal((64, 5))
    parts = S.partition(64, 3)
    fakes = [FakeSlab(glob, y0, n) for y0, n in parts]

    class Buf:
        def __init__(self):
            self.v = None

        def data_ptr(self):
            return self

    class Dev:
        def __init__(self, f):
            self.f = f

        def halo_bytes(self):
            return S.GHOST * 5 * 8

        def pack(self, side, buf, nbytes, device):
            buf.v = self.f.a[self.f.rows(side, False)].copy()

        def unpack(self, side, buf, nbytes, device):
            self.f.a[self.f.rows(side, True)] = buf.v

    bufs = [(Buf(), Buf()) for _ in fakes]
    S.exchange_local([Dev(f) for f in fakes], bufs)
    for f in fakes:
        assert np.array_equal(f.a, glob[f.glob_rows])
