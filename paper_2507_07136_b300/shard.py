"""Sharding of a many-view batch across ranks (one process per GPU).

Views are independent given the replicated scene, so a batch of views shards with no collective
on the data path: each rank renders and queries its own views.  The partition balances the
pixel count (the splat and the relevancy scale with pixels) by the longest-processing-time rule:
views in decreasing pixel count, each to the rank with the fewest pixels so far (lowest rank on a
tie), which keeps the largest load within 4/3 of the optimum.  Every rank computes the same
partition from the view sizes alone.
"""
from __future__ import annotations


def partition_views(pixels: list[int], world: int) -> list[list[int]]:
    """View indices per rank (each list ascending), balanced by pixel count."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(pixels)), key=lambda v: (-int(pixels[v]), v))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for v in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(v)
        load[r] += int(pixels[v])
    return [sorted(p) for p in parts]


def rank_views(pixels: list[int], rank: int, world: int) -> list[int]:
    """The views of one rank."""
    return partition_views(pixels, world)[rank]
