"""Host-side work split for runs with one process per GPU.

One ID either runs as replicas (every rank its own Philox problem id, no
collective on the data path) or, with its rows split across shards, as the
row-sharded block loop of sharded_id(): per block a merge of the shards'
candidate lists, an exchange of the candidate rows and one sum of ||d||_1.  A list of independent problems (the batched form) is cut into
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

    With rows split across ranks, each rank ranks the race keys of Alg. 2's
    sampling step over its own rows (keys drawn with the global row ids as
    Philox counters) and contributes its b smallest; the global b smallest are
    among those.  keys, rows: sequences of per-rank arrays (any order).  Returns the
    rows of the b smallest pairs in ascending (key, row) order, the order of
    S_t of one process.
    """
    import numpy as np
    k = np.concatenate([np.asarray(x, dtype=np.float64) for x in keys]) if len(keys) else np.zeros(0)
    r = np.concatenate([np.asarray(x, dtype=np.int64) for x in rows]) if len(rows) else np.zeros(0, np.int64)
    order = np.lexsort((r, k))
    return r[order[:int(b)]]


# ---------------------------------------------------------------- the row-sharded block loop
class LocalComm:
    """All shards in this process: the exchanges are plain list operations."""

    def allgather(self, obj):
        return [obj]

    def allreduce_sum(self, x):
        return x


class DistComm:
    """One or more shards per process, exchanged over the default torch.distributed group
    (gloo or NCCL); object all-gathers for the candidate lists, sums for the rest."""

    def allgather(self, obj):
        import torch.distributed as dist
        out = [None] * dist.get_world_size()
        dist.all_gather_object(out, obj)
        return out

    def allreduce_sum(self, x):
        import numpy as np
        import torch
        import torch.distributed as dist
        t = torch.as_tensor(np.asarray(x, dtype=np.float64)).clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy() if t.dim() else float(t.item())


def sharded_id(shards, tol, block, k_cap, comm=None):
    """RBRP (Alg. 2, then Alg. 3) of one ID whose rows are split into shards.

    shards: this process's shards, objects with sum_sq, d and the methods draw(),
    rows(S_t), block(V, S_t), l_rows(S, k), w(L1, S) (paper_2309_16002_gb300.rbrp.Shard,
    or a stand-in with the same contract); comm: LocalComm() when every shard is in this
    process, DistComm() with one group member per process.  tol: tau of the stopping test
    (< 0: fixed rank k_cap).  Per block: each shard draws its candidates with global row
    ids, the lists are merged to the global S_t (merge_candidates), the candidate rows are
    assembled from their owners, every shard runs the rest of the block on the same V,
    and ||d||_1 is summed.  Returns dict(S, W (one per local shard), k, blocks,
    rel_err_sq, d0, d_final).
    """
    import numpy as np
    comm = comm or LocalComm()
    d = shards[0].d
    D0 = float(comm.allreduce_sum(sum(sh.sum_sq for sh in shards)))
    D = D0
    S = []
    blocks = 0
    while len(S) < k_cap and (tol < 0 or D > tol * D0):
        local = [sh.draw() for sh in shards]
        every = [c for part in comm.allgather(local) for c in part]
        b_t = min(int(block), k_cap - len(S), sum(len(rows) for rows, _ in every))
        if b_t <= 0:
            break
        S_t = merge_candidates([keys for _, keys in every], [rows for rows, _ in every], b_t)
        V = np.zeros((b_t, d))
        for sh in shards:
            part, own = sh.rows(S_t)
            V[own] = part[own]
        V = np.asarray(comm.allreduce_sum(V)).reshape(b_t, d)  # each row comes from exactly one shard
        results = [sh.block(V, S_t) for sh in shards]
        acc = results[0][0]
        for other, _ in results[1:]:
            if not np.array_equal(other, acc):
                raise RuntimeError("shards accepted different rows: their inputs differ")
        D = float(comm.allreduce_sum(sum(r[1] for r in results)))
        blocks += 1
        if len(acc) == 0:
            break
        S.extend(int(x) for x in acc)
    k = len(S)
    S = np.array(S, dtype=np.int64)
    L1 = np.zeros((k, k))
    for sh in shards:
        part, own = sh.l_rows(S, k)
        L1[own] = part[own]
    L1 = np.asarray(comm.allreduce_sum(L1)).reshape(k, k)
    W = [sh.w(L1, S) for sh in shards]
    return dict(S=S, W=W, k=k, blocks=blocks, d0=D0, d_final=D, rel_err_sq=(D / D0) if D0 > 0 else 0.0)
