"""Multi-process host logic on CPU ranks (torch.distributed, gloo, world size 2).

Covers what a run with one process per GPU does on the host:
  * contiguous, cost-balanced shards of a list of independent problems, with
    the shard's first index as Philox problem-id base, reproduce one call over
    the whole list (the batched form split across ranks, no exchange);
  * max-over-ranks timing;
  * the row-sharded form of the block loop of Alg. 2 (rows split across ranks,
    race keys drawn with global row ids, a global top-b_t merge of per-rank
    candidates, the candidate rows all-gathered, the filter replicated, the
    residual update local, ||d||_1 all-reduced) selects the same skeletons as
    one process.  The steps are the oracle's; only the distribution is new.
Nothing here touches a GPU.
"""

import os
import socket
import sys
from datetime import timedelta

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import philox  # noqa: E402
from oracle import rbrp as O  # noqa: E402
from paper_2309_16002_gb300 import shard  # noqa: E402
from paper_2309_16002_gb300 import workloads as WL  # noqa: E402

WORLD = 2


def _free_port():
    s = socket.socket(socket.AF_INET, socket.SOCK_STREAM)
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
    return dist


def _batch_problems():
    return WL.kernel_blocks(P=7, m_range=(24, 90), n_range=(10, 30), seed=11, dtype=np.float64)


def _worker_batched(rank, world, port, out_dir):
    dist = _init(rank, world, port)
    try:
        Xs = _batch_problems()
        costs = [shard.problem_cost(*X.shape) for X in Xs]
        lo, hi = shard.my_shard(costs, world, rank)
        # every rank computes the same cuts
        cuts = [None] * world
        dist.all_gather_object(cuts, shard.shard_bounds(costs, world))
        assert all(c == cuts[0] for c in cuts)
        mine = {}
        for j, X in enumerate(Xs[lo:hi]):
            r = O.rbrp_id(X, tau=1e-6, b=4, seed=3, problem=lo + j)
            mine[lo + j] = (r["S"].tolist(), r["rel_err_sq"])
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        t = shard.max_over_ranks(1.5 + rank)
        tot = shard.sum_over_ranks(hi - lo)
        if rank == 0:
            merged = {}
            for p in parts:
                merged.update(p)
            np.save(os.path.join(out_dir, "batched.npy"),
                    np.array([merged, t, tot, cuts[0]], dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _sharded_rbrp(dist, rank, world, X, tau, b, seed, problem):
    """Alg. 2 with the rows of X split across ranks; returns (S, D, D0) on every rank."""
    import torch
    n, dim = X.shape
    lo, hi = shard.shard_bounds([1] * n, world)[rank]
    R = np.array(X[lo:hi], dtype=np.float64)
    rows = np.arange(lo, hi, dtype=np.int64)
    in_S = np.zeros(hi - lo, dtype=bool)
    d = O.row_sq_norms(R)

    def allsum(x):
        tt = torch.tensor([float(x)], dtype=torch.float64)
        dist.all_reduce(tt)
        return float(tt.item())

    def allgather(obj):
        out = [None] * world
        dist.all_gather_object(out, obj)
        return out

    D0 = allsum(d.sum())
    D = D0
    Q = np.zeros((dim, 0))
    S = []
    t = 0
    while len(S) < min(n, dim) and D > tau * D0:
        eligible = (~in_S) & (d > 0)
        b_t = min(b, int(allsum(eligible.sum())), min(n, dim) - len(S))
        if b_t <= 0:
            break
        t += 1
        # local race keys with global row ids as Philox counters, local top-b_t
        u = philox.uniforms(rows.astype(np.uint64), t, seed, problem)
        kappa = np.full(hi - lo, np.inf)
        kappa[eligible] = -np.log(u[eligible]) / d[eligible]
        loc = np.lexsort((rows, kappa))[:b_t]
        loc = loc[np.isfinite(kappa[loc])]
        cand = allgather((kappa[loc], rows[loc]))
        S_t = shard.merge_candidates([c[0] for c in cand], [c[1] for c in cand], b_t)
        # owners contribute the sampled rows
        own = {int(i): R[int(i) - lo] for i in S_t if lo <= int(i) < hi}
        got = {}
        for g in allgather(own):
            got.update(g)
        V = np.stack([got[int(i)] for i in S_t], axis=1)
        for _ in range(2):
            V = V - Q @ (Q.T @ V)
        QV, RV, piv, _ = O.cpqr(V)
        bp, _ = O.filter_rank(RV, 1.0 / b_t)
        if bp == 0:
            break
        Sp = S_t[piv[:bp]]
        Qp = QV[:, :bp]
        Q = np.concatenate([Q, Qp], axis=1)
        active = ~in_S
        Lhat = np.zeros((hi - lo, bp))
        Lhat[active] = R[active] @ Qp
        S.extend(int(s) for s in Sp)
        mine = np.array([int(s) - lo for s in Sp if lo <= int(s) < hi], dtype=np.int64)
        in_S[mine] = True
        R[active] -= Lhat[active] @ Qp.T
        R[mine] = 0.0
        d = O.row_sq_norms(R)
        d[in_S] = 0.0
        D = allsum(d.sum())
    return S, D, D0


def _worker_rows(rank, world, port, out_dir):
    dist = _init(rank, world, port)
    try:
        X = WL.gmm_pitfall(n=312, d=60, k=12, seed=6)
        S, D, D0 = _sharded_rbrp(dist, rank, world, X, 1e-3, 8, 0, 2)
        res = [None] * world
        dist.all_gather_object(res, (S, D, D0))
        if rank == 0:
            np.save(os.path.join(out_dir, "rows.npy"), np.array(res, dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _spawn(fn, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(fn, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD, join=True)


def test_shard_bounds_cover_and_balance():
    costs = [5, 1, 1, 1, 10, 2]
    assert shard.shard_bounds(costs, 2) == [(0, 4), (4, 6)]
    assert shard.shard_bounds([1] * 7, 3) == [(0, 2), (2, 5), (5, 7)]
    assert shard.shard_bounds([], 2) == [(0, 0), (0, 0)]
    rng = np.random.default_rng(0)
    for _ in range(50):
        P = int(rng.integers(0, 40))
        w = int(rng.integers(1, 9))
        c = rng.integers(0, 1000, size=P).tolist()
        b = shard.shard_bounds(c, w)
        assert len(b) == w and b[0][0] == 0 and b[-1][1] == P
        assert all(b[r][1] == b[r + 1][0] and b[r][0] <= b[r][1] for r in range(w - 1))
        if P and sum(c):
            worst = max(sum(c[lo:hi]) for lo, hi in b)
            assert worst <= sum(c) / w + max(c)
    with pytest.raises(ValueError):
        shard.shard_bounds([1], 0)
    with pytest.raises(ValueError):
        shard.my_shard([1], 2, 2)


def test_merge_candidates_order_and_ties():
    keys = [np.array([0.5, 0.1, 0.3]), np.array([0.1, 0.2])]
    rows = [np.array([4, 7, 1]), np.array([2, 9])]
    assert shard.merge_candidates(keys, rows, 3).tolist() == [2, 7, 9]
    assert shard.merge_candidates(keys, rows, 10).tolist() == [2, 7, 9, 1, 4]


def test_gloo_batched_shards_match_one_call(tmp_path):
    _spawn(_worker_batched, tmp_path)
    merged, t, tot, cuts = np.load(tmp_path / "batched.npy", allow_pickle=True)
    Xs = _batch_problems()
    assert t == 1.5 + (WORLD - 1)
    assert tot == len(Xs)
    assert sorted(merged) == list(range(len(Xs)))
    assert all(lo < hi for lo, hi in cuts)  # both ranks got work
    for p, X in enumerate(Xs):
        r = O.rbrp_id(X, tau=1e-6, b=4, seed=3, problem=p)
        S, e = merged[p]
        assert S == r["S"].tolist()
        assert e == r["rel_err_sq"]


def test_gloo_row_sharded_block_loop_matches_one_process(tmp_path):
    _spawn(_worker_rows, tmp_path)
    res = np.load(tmp_path / "rows.npy", allow_pickle=True)
    S0, D0_, Dinit = res[0]
    for S, D, Di in res[1:]:
        assert S == S0 and D == D0_ and Di == Dinit  # every rank holds the same result
    X = WL.gmm_pitfall(n=312, d=60, k=12, seed=6)
    ref = O.rbrp(X, tau=1e-3, b=8, seed=0, problem=2)
    assert S0 == ref["S"].tolist()
    assert abs(D0_ - ref["D"]) <= 1e-9 * ref["D0"]
    assert abs(Dinit - ref["D0"]) <= 1e-12 * ref["D0"]
