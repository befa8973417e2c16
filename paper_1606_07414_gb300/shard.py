"""Sharding a list of images over ranks (one process per GPU).

Blocks and images are independent (Sec. 3.1 codes each 16x16 block on its
own), so a job over several GPUs needs no exchange: each rank codes a subset
of whole images and the results are the union.  ``shard_images`` gives every
rank the same deterministic assignment from the images' block counts alone,
so the ranks agree without communicating.
"""
from __future__ import annotations

from typing import Sequence


def shard_images(blocks: Sequence[int], world: int) -> list[list[int]]:
    """Assign image i (of blocks[i] blocks) to one of `world` ranks.

    Longest-processing-time greedy: images in decreasing block count (ties by
    index) go to the rank with the fewest blocks so far (ties to the lowest
    rank).  Every image lands on exactly one rank, and the busiest rank holds
    at most the mean plus the largest image.  Returns, per rank, its image
    indices in increasing order."""
    if world < 1:
        raise ValueError("world must be at least 1")
    if any(int(b) < 0 for b in blocks):
        raise ValueError("block counts must be non-negative")
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(blocks)), key=lambda j: (-int(blocks[j]), j)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(blocks[i])
    return [sorted(s) for s in out]


def rank_images(blocks: Sequence[int], rank: int, world: int) -> list[int]:
    """The image indices rank `rank` codes (see shard_images)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return shard_images(blocks, world)[rank]
