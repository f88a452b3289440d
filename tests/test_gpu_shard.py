"""Row shards of one ID on the GPU (include/rbrp.h, rbrp_shard_*): the shards of one ID run
one after the other on one GPU through the C ABI, driven by shard.sharded_id, and must
reproduce one unsharded rbrp_id call -- the same skeletons bit for bit (FP64), the same W
rows (up to the W solve's blocking) and ||d||_1 up to the order of the final sum.

Shards of at least 40000 rows keep every product of the block loop in the same
summation order as the unsharded call (one K split at these sizes), so their residual rows
are bitwise those of one call; with smaller, uneven shards the skeletons are checked
against the oracle under the per-block near-tie rule instead."""
import numpy as np
import pytest

from oracle import parity as P
from oracle import rbrp as O
from paper_2309_16002_gb300 import shard
from paper_2309_16002_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2309_16002_gb300 import rbrp
    rbrp.load()
    return rbrp


def _shards(G, X, cuts, k_cap, **kw):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0")
    return [G.Shard(Xd[lo:hi], lo, k_cap, **kw) for lo, hi in cuts]


def test_two_shards_reproduce_one_call_fp64(G):
    import torch
    X, _ = WL.spectral(n=80000, d=100, rate=0.9, seed=51)
    kc = min(X.shape)
    sh = _shards(G, X, [(0, 40000), (40000, 80000)], kc, block=16, seed=7, precision="fp64")
    out = shard.sharded_id(sh, 1e-6, 16, kc)
    one = G.rbrp_id(torch.from_numpy(X).to("cuda:0"), 1e-6, block=16, seed=7, precision="fp64")
    S1 = one["S"].cpu().numpy()
    assert out["S"].tolist() == S1.tolist()
    W = torch.cat(out["W"], dim=0).cpu().numpy()
    W1 = one["W"].cpu().numpy()
    assert np.max(np.abs(W - W1)) <= 1e-10 * max(1.0, np.max(np.abs(W1)))
    assert abs(out["rel_err_sq"] - one["rel_err_sq"]) <= 1e-12 * one["rel_err_sq"]
    assert np.array_equal(W[out["S"]], np.eye(out["k"]))


def test_uneven_shards_match_the_oracle(G):
    """Three uneven shards (one smaller than b) of a 5000 x 80 problem, FP64: the oracle's
    skeletons under the near-tie rule, and its error within 1e-10."""
    import torch
    X, _ = WL.spectral(n=5000, d=80, rate=0.88, seed=52)
    kc = min(X.shape)
    sh = _shards(G, X, [(0, 2990), (2990, 3000), (3000, 5000)], kc, block=16, seed=3, precision="fp64")
    out = shard.sharded_id(sh, 1e-6, 16, kc)
    ref = O.rbrp_id(X, tau=1e-6, b=16, seed=3)
    ok, note = P.fp64_skeleton_check(ref, out["S"], 1e-6)
    assert ok, note
    W = torch.cat(out["W"], dim=0).cpu().numpy()
    if not note:
        assert abs(P.id_error(X, out["S"], W) - P.id_error(X, ref["S"], ref["W"])) <= 1e-10


def test_shards_with_tensor_core_update(G):
    """TF32 update with the FP64 chain on two shards: the literal mixed bar against the oracle."""
    import torch
    X = WL.zipf_gmm(n=20000, d=300, clusters=40, seed=2)
    kc = min(X.shape)
    sh = _shards(G, X, [(0, 12000), (12000, 20000)], kc, block=64, seed=0, precision="tf32", chain="fp64")
    out = shard.sharded_id(sh, 1e-3, 64, kc)
    ref = O.rbrp_id(X, tau=1e-3, b=64, seed=0)
    W = torch.cat(out["W"], dim=0).cpu().numpy()
    e_gpu, e_ref = P.id_error(X, out["S"], W), P.id_error(X, ref["S"], ref["W"])
    assert P.mixed_bar(e_gpu, e_ref), (e_gpu, e_ref)
    assert np.array_equal(W[out["S"]], np.eye(out["k"]))


def test_shard_argument_checks(G):
    import torch
    X = torch.zeros((100, 10), dtype=torch.float64, device="cuda:0")
    with pytest.raises(G.RBRPError):
        G.Shard(X, 0, 11, block=4)                         # k_cap > d
    with pytest.raises(G.RBRPError):
        G.Shard(X.float(), 0, 10, block=4, precision="tf32")  # the FP32 chain has no shard form
