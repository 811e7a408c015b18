"""Splitting a tile list across GPUs. Tiles are independent (the paper cuts
slides into independent 4K x 4K tiles, Section 5), so every GPU runs its own
process on its own share and no data crosses between GPUs: replicas only.
Shares are balanced by pixel count, longest tile first."""
from __future__ import annotations


def lpt_shards(sizes, world: int):
    """Indices of the tiles of each of `world` shards: tiles in decreasing
    H*W order, each to the shard with the fewest pixels so far (ties to the
    lowest shard). sizes: list of (H, W)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i))
    load = [0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        k = min(range(world), key=lambda j: (load[j], j))
        shards[k].append(i)
        load[k] += sizes[i][0] * sizes[i][1]
    return [sorted(s) for s in shards]
