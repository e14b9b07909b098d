"""Sharding of the many-view batch across ranks (CPU only): the partition and, with two gloo
ranks, that every rank derives the same complete, disjoint partition and that the batch time is
the maximum over ranks (the host logic of a multi-GPU run of the batched workload)."""
import os
import socket

import pytest

import lsv2_synth as syn
from paper_2507_07136_b300.shard import partition_views, rank_views

torch = pytest.importorskip("torch")


def batched_pixels():
    return [w * h for w, h in syn.BATCH_RESOLUTIONS]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 16, 20])
def test_partition_covers_every_view_once_and_balances(world):
    px = batched_pixels()
    parts = partition_views(px, world)
    assert len(parts) == world
    flat = sorted(v for p in parts for v in p)
    assert flat == list(range(len(px)))
    loads = [sum(px[v] for v in p) for p in parts]
    # longest-processing-time bound: the largest load is within max view of the smallest
    assert max(loads) - min(loads) <= max(px)
    assert max(loads) <= 4 / 3 * max(sum(px) / world, max(px)) + 1
    assert parts == partition_views(px, world)          # deterministic


def test_partition_of_equal_views_is_round_robin_by_size_then_index():
    assert partition_views([10, 10, 10, 10], 2) == [[0, 2], [1, 3]]
    assert partition_views([5, 40, 5, 40], 2) == [[0, 1], [2, 3]]   # 1, 3, then 0 (tie: rank 0), 2
    with pytest.raises(ValueError):
        partition_views([1], 0)


def _worker(rank, world, port, px):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = rank_views(px, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    assert sorted(v for p in got for v in p) == list(range(len(px)))
    assert got == partition_views(px, world)
    # each rank's "batch time" grows with its pixels; the job time is the maximum
    t = torch.tensor([float(sum(px[v] for v in mine))])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    assert t.item() == max(sum(px[v] for v in p) for p in got)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_shards():
    import torch.multiprocessing as mp
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    mp.start_processes(_worker, args=(2, _free_port(), batched_pixels()), nprocs=2, join=True, start_method="spawn")
