"""Host-side work split for runs with one process per GPU.

One ID exchanges nothing between processes here: every rank runs its own
replica (its own Philox problem id), so there is no collective on the data
path.  A list of independent problems (the batched form) is cut into
contiguous shards of about equal work, one per rank; shard r passes the index
of its first problem as the Philox problem-id base, so every problem draws the
same skeletons whichever shard solves it and the union of the shards' results
equals one call over the whole list.  Timing is reduced as the maximum over
ranks.  Nothing here touches a GPU.
"""

from __future__ import annotations


def problem_cost(m: int, n: int) -> int:
    """Work of one m x n problem, in elements of one pass over it."""
    return int(m) * int(n)


def shard_bounds(costs, world: int):
    """Contiguous shards [lo, hi) of the problems, one per rank.

    The cut before rank r is the index whose prefix cost is closest to
    r / world of the total (the earlier index on a tie; integer arithmetic, so
    every rank computes the same cuts without communicating).  Shards may be
    empty when there are fewer problems than ranks.
    """
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [int(c) for c in costs]
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    total = sum(costs)
    P = len(costs)
    cuts = [0]
    prefix, i = 0, 0
    for r in range(1, world):
        target = total * r  # prefix * world is compared with total * r in integers
        while i < P and (prefix + costs[i]) * world <= target:
            prefix += costs[i]
            i += 1
        if i < P and abs((prefix + costs[i]) * world - target) < abs(prefix * world - target):
            prefix += costs[i]
            i += 1
        cuts.append(max(i, cuts[-1]))
    cuts.append(P)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def my_shard(costs, world: int, rank: int):
    """(lo, hi) of this rank's shard."""
    if not 0 <= int(rank) < int(world):
        raise ValueError("rank out of range")
    return shard_bounds(costs, world)[int(rank)]


def replica_problem_id(rank: int, base: int = 0) -> int:
    """Philox problem id of rank r's replica of the single ID."""
    return int(base) + int(rank)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank number over the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def merge_candidates(keys, rows, b: int):
    """Global selection of the b smallest (key, row) pairs from per-rank candidate lists.

    With rows split across ranks, each rank ranks the race keys of Alg. 2 line
    5 over its own rows (keys drawn with the global row ids as Philox
    counters) and contributes its b smallest; the global b smallest are among
    those.  keys, rows: sequences of per-rank arrays (any order).  Returns the
    rows of the b smallest pairs in ascending (key, row) order, the order of
    S_t of one process.
    """
    import numpy as np
    k = np.concatenate([np.asarray(x, dtype=np.float64) for x in keys]) if len(keys) else np.zeros(0)
    r = np.concatenate([np.asarray(x, dtype=np.int64) for x in rows]) if len(rows) else np.zeros(0, np.int64)
    order = np.lexsort((r, k))
    return r[order[:int(b)]]
