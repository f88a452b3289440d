"""Multi-process host logic on CPU ranks (torch.distributed, gloo, world size 2).

Covers what a run with one process per GPU does on the host:
  * contiguous, cost-balanced shards of a list of independent problems, with
    the shard's first index as Philox problem-id base, reproduce one call over
    the whole list (the batched form split across ranks, no exchange);
  * max-over-ranks timing;
  * the row-sharded form of the block loop of Alg. 2 (shard.sharded_id over
    torch.distributed: rows split across ranks, race keys drawn with global row
    ids, a global top-b_t merge of per-rank candidates, the candidate rows
    exchanged, the filter replicated, the residual update local, ||d||_1
    summed) selects the same skeletons as one process.  The shards here are an
    oracle-backed stand-in for the GPU shards behind the same contract.
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


class OracleShard:
    """Rows [lo, hi) of X with the oracle's FP64 steps behind the shard contract of
    paper_2309_16002_gb300.shard.sharded_id (draw / rows / block / l_rows / w): a CPU
    stand-in for a GPU shard, so that the exchange logic runs on gloo ranks."""

    def __init__(self, X, lo, hi, k_cap, b, seed, problem):
        self.R = np.array(X[lo:hi], dtype=np.float64)
        self.lo, self.hi, self.n, self.d = lo, hi, hi - lo, X.shape[1]
        self.rows_g = np.arange(lo, hi, dtype=np.int64)
        self.k_cap, self.b, self.seed, self.problem = k_cap, b, seed, problem
        self.dv = O.row_sq_norms(self.R)
        self.sum_sq = float(self.dv.sum())
        self.in_S = np.zeros(self.n, dtype=bool)
        self.Q = np.zeros((self.d, 0))
        self.L = np.zeros((self.n, 0))
        self.t = 0
        self.k = 0

    def draw(self):
        eligible = (~self.in_S) & (self.dv > 0)
        b_t = min(self.b, int(eligible.sum()), self.k_cap - self.k)
        u = philox.uniforms(self.rows_g.astype(np.uint64), self.t + 1, self.seed, self.problem)
        kappa = np.full(self.n, np.inf)
        kappa[eligible] = -np.log(u[eligible]) / self.dv[eligible]
        loc = np.lexsort((self.rows_g, kappa))[:max(b_t, 0)]
        return self.rows_g[loc], kappa[loc]

    def rows(self, S_t):
        own = (S_t >= self.lo) & (S_t < self.hi)
        V = np.zeros((len(S_t), self.d))
        V[own] = self.R[S_t[own] - self.lo]
        return V, own

    def block(self, V, S_t):
        self.t += 1
        Vt = O.project_out(np.array(V).T, self.Q, 2)
        QV, RV, piv, _ = O.cpqr(Vt)
        bp, _ = O.filter_rank(RV, 1.0 / len(S_t))
        if bp == 0:
            return np.zeros(0, dtype=np.int64), float(self.dv.sum())
        Sp = np.asarray(S_t)[piv[:bp]]
        Qp = QV[:, :bp]
        self.Q = np.concatenate([self.Q, Qp], axis=1)
        active = ~self.in_S
        Lhat = np.zeros((self.n, bp))
        Lhat[active] = self.R[active] @ Qp
        mine = np.array([int(s) - self.lo for s in Sp if self.lo <= int(s) < self.hi], dtype=np.int64)
        self.in_S[mine] = True
        self.L = np.concatenate([self.L, Lhat], axis=1)
        self.R[active] -= Lhat[active] @ Qp.T
        self.R[mine] = 0.0
        self.dv = O.row_sq_norms(self.R)
        self.dv[self.in_S] = 0.0
        self.k += bp
        return Sp.astype(np.int64), float(self.dv.sum())

    def l_rows(self, S, k):
        own = (S >= self.lo) & (S < self.hi)
        out = np.zeros((len(S), k))
        out[own] = self.L[S[own] - self.lo, :k]
        return out, own

    def w(self, L1, S):
        import scipy.linalg as sla
        W = sla.solve_triangular(L1.T, self.L[:, :len(S)].T, lower=False).T if len(S) else np.zeros((self.n, 0))
        for j, s in enumerate(S):
            if self.lo <= s < self.hi:
                W[s - self.lo] = 0.0
                W[s - self.lo, j] = 1.0
        return W


def _worker_rows(rank, world, port, out_dir):
    dist = _init(rank, world, port)
    try:
        X = WL.gmm_pitfall(n=312, d=60, k=12, seed=6)
        lo, hi = shard.shard_bounds([1] * X.shape[0], world)[rank]
        sh = OracleShard(X, lo, hi, min(X.shape), 8, 0, 2)
        out = shard.sharded_id([sh], 1e-3, 8, min(X.shape), comm=shard.DistComm())
        res = [None] * world
        dist.all_gather_object(res, (out["S"].tolist(), out["d_final"], out["d0"], lo, out["W"][0]))
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
    """The product's row-sharded driver (shard.sharded_id over torch.distributed) on two gloo
    ranks, each holding half of the rows behind the shard contract, selects the skeletons of
    one unsharded oracle run; each rank's rows of W are those of the unsharded W."""
    _spawn(_worker_rows, tmp_path)
    res = np.load(tmp_path / "rows.npy", allow_pickle=True)
    S0, D0_, Dinit = res[0][0], res[0][1], res[0][2]
    for S, D, Di, _, _ in res[1:]:
        assert S == S0 and D == D0_ and Di == Dinit  # every rank holds the same result
    X = WL.gmm_pitfall(n=312, d=60, k=12, seed=6)
    ref = O.rbrp_id(X, tau=1e-3, b=8, seed=0, problem=2)
    assert S0 == ref["S"].tolist()
    assert abs(D0_ - ref["D"]) <= 1e-9 * ref["D0"]
    assert abs(Dinit - ref["D0"]) <= 1e-12 * ref["D0"]
    W = np.concatenate([r[4] for r in sorted(res, key=lambda r: r[3])], axis=0)
    assert np.allclose(W, ref["W"], atol=1e-10)
