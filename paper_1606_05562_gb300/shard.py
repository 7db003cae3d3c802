"""Host logic for running the path on several GPUs (one process per GPU).

Every 16x16 block is independent (Sec. 4: the procedure is repeated for each
block), so images are the natural unit of work: each rank compresses a
disjoint set of whole images and no data-path collective is needed.  Only
the per-image results (PSNR, SSE) are gathered, on the host.
"""

from __future__ import annotations

import heapq


def contiguous_shard(n_items: int, world: int, rank: int) -> range:
    """Balanced contiguous range of item indices for ``rank``."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def balanced_shards(pixel_counts, world: int) -> list:
    """Assign items of uneven size to ranks, largest first onto the least
    loaded rank (LPT).  Returns one sorted index list per rank; ties go to the
    lowest rank, so the assignment is deterministic."""
    if world < 1:
        raise ValueError("bad world")
    order = sorted(range(len(pixel_counts)), key=lambda i: (-pixel_counts[i], i))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + pixel_counts[i], r))
    return [sorted(s) for s in shards]


def merge_results(per_rank_indices, per_rank_values, n_items: int) -> list:
    """Scatter per-rank results back into item order; every item exactly once."""
    out = [None] * n_items
    for idx, vals in zip(per_rank_indices, per_rank_values):
        if len(idx) != len(vals):
            raise ValueError("result count mismatch")
        for i, v in zip(idx, vals):
            if out[i] is not None:
                raise ValueError(f"item {i} assigned twice")
            out[i] = v
    missing = [i for i, v in enumerate(out) if v is None]
    if missing:
        raise ValueError(f"items without a result: {missing[:5]}")
    return out
