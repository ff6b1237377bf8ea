"""Frame sharding across processes (one process per GPU).

Every pixel is independent given its line's analytic signal and frames are independent, so the
path shards by frames with no data exchange: each rank demodulates its own frames through its own
context. ``shard_frames`` assigns frames to ranks balancing pixel counts (longest processing time
first, ties to the lower rank), deterministically, so every rank computes the same assignment
without communicating."""
from __future__ import annotations

from typing import Sequence


def shard_frames(shapes: Sequence[tuple[int, int]], world: int) -> list[list[int]]:
    """Frame indices per rank, balanced by pixels; each list is in increasing frame order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    order = sorted(range(len(shapes)), key=lambda i: (-shapes[i][0] * shapes[i][1], i))
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += shapes[i][0] * shapes[i][1]
    return [sorted(p) for p in parts]


def my_frames(shapes: Sequence[tuple[int, int]], rank: int, world: int) -> list[int]:
    return shard_frames(shapes, world)[rank]
