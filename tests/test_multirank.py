"""Host logic of the multi-GPU (N > 1) bench path, run as two gloo ranks on CPU.

The path shards as independent runs (one per rank, weak scaling, no data-path
collective): each rank gets its own seed, the timed region is the slowest
rank's, and the reported value is the updates of all ranks over that time.
"""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = 1.0 + 0.5 * rank          # rank 1 is the slower one
    t = bench.max_over_ranks(local_seconds, dist, device="cpu")
    seed = bench.replica_seed(0, rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    value = bench.aggregate_glups(world, 4096 * 4096, 10, t)
    out[rank] = (t, tuple(seeds), value)
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, seeds, value = res[rank]
        assert t == 1.5                          # max over ranks
        assert len(set(seeds)) == 2              # independent replicas
        assert value == pytest.approx(2 * 4096 * 4096 * 10 / 1.5 / 1e9)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.replica_seed(7, 0) == 7
