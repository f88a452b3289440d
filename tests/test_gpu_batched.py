"""GPU parity of the batched entry point (rbrp_id_batched, one launch for P problems).

Problem p of a batch uses Philox problem id (base + p), base 0 unless given, so it must
reproduce the single-problem oracle run with that problem id.  Bars, problem by problem (as in test_gpu_parity):
  FP64  skeleton indices identical to the oracle's (or a near-tie the oracle logged at the
        first block where the runs part, oracle/parity.py) and |e_gpu - e_oracle| <= 1e-10,
        e = ||X - W X_S||_F / ||X||_F;
  FP32  e_gpu <= max(1.05 e_oracle, e_oracle + 1e-5) against the oracle's own run of the
        problem, the same bar against the exact error of the GPU's skeletons (W = X X_S^+),
        e_gpu^2 <= 1.05 tol, k <= 1.1 k_oracle + b.
W(S, :) = I exactly in both.
"""
import numpy as np
import pytest

from oracle import parity as P
from oracle import rbrp as O
from paper_2309_16002_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _skeletons_ok(ref, S, tau, where):
    ok, note = P.fp64_skeleton_check(ref, S, tau)
    assert ok, (where, note)
    if note:
        print("near-tie excuse (%s): %s" % (where, note))
    return not note


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


def _problems(dtype):
    """Kernel blocks of the batched workload's kind (smaller), plus edge cases."""
    rng = np.random.default_rng(41)
    Xs = [WL.kernel_block(rng, m, n, dtype=np.float32).astype(dtype)
          for m, n in [(64, 32), (200, 48), (333, 64), (97, 256), (130, 33), (600, 200)]]
    Xs.append((rng.standard_normal((150, 3)) @ rng.standard_normal((3, 40))).astype(dtype))  # exact rank 3
    Xs.append(np.zeros((70, 20), dtype=dtype))                                               # D0 = 0
    Xs.append(np.repeat(rng.standard_normal((8, 30)), 12, axis=0).astype(dtype))             # duplicated rows
    Xs.append(rng.standard_normal((20, 50)).astype(dtype))                                   # m < n
    Xs.append(rng.standard_normal((1, 16)).astype(dtype))                                    # one row
    Xs.append(rng.standard_normal((40, 1)).astype(dtype))                                    # one column
    return Xs


def _run(G, Xs, tol, **kw):
    import torch
    Xd = [torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0") for X in Xs]
    outs = G.rbrp_id_batched(Xd, tol, **kw)
    for o in outs:
        o["S"] = o["S"].cpu().numpy()
        o["W"] = o["W"].cpu().numpy()
    return outs


def _e(X, S, W):
    return P.id_error(X, S, W)


@pytest.mark.parametrize("tol,b", [(1e-5, 16), (1e-9, 8)])
def test_batched_fp64_matches_oracle(G, tol, b):
    Xs = _problems(np.float64)
    outs = _run(G, Xs, tol, block=b, seed=7, precision="fp64")
    for p, (X, out) in enumerate(zip(Xs, outs)):
        ref = O.rbrp_id(X, tau=tol, b=b, seed=7, problem=p)
        S = out["S"].tolist()
        assert out["status"] in (0, 5), (p, out["status"])
        if not _skeletons_ok(ref, S, tol, p):
            continue
        k = len(S)
        assert np.array_equal(out["W"][out["S"]], np.eye(k)), p
        if k:
            assert abs(_e(X, out["S"], out["W"]) - _e(X, ref["S"], ref["W"])) <= 1e-10, p
        assert abs(out["rel_err_sq"] - ref["rel_err_sq"]) <= 1e-10 * max(1.0, ref["rel_err_sq"]) + 1e-13, p


@pytest.mark.parametrize("tol,b", [(1e-5, 16), (1e-4, 32)])
def test_batched_fp32_bar(G, tol, b):
    Xs = _problems(np.float32)
    outs = _run(G, Xs, tol, block=b, seed=3, precision="fp32")
    for p, (X, out) in enumerate(zip(Xs, outs)):
        X64 = X.astype(np.float64)
        k = len(out["S"])
        assert out["status"] in (0, 5), (p, out["status"])
        assert np.array_equal(out["W"][out["S"]], np.eye(k)), p
        assert len(set(out["S"].tolist())) == k, p
        if not np.any(X64):
            assert k == 0
            continue
        ref = O.rbrp_id(X64, tau=tol, b=b, seed=3, problem=p)
        e_gpu = _e(X64, out["S"], out["W"])
        e_ref = _e(X64, ref["S"], ref["W"])
        assert P.mixed_bar(e_gpu, e_ref), (p, e_gpu, e_ref)
        e_same = float(np.sqrt(O.skeleton_error_sq(X64, out["S"])))
        assert P.mixed_bar(e_gpu, e_same), (p, e_gpu, e_same)
        if out["status"] == 0:
            assert e_gpu ** 2 <= 1.05 * tol + 1e-10, (p, e_gpu ** 2, tol)
        assert k <= 1.1 * len(ref["S"]) + b, (p, k, len(ref["S"]))


def test_batched_fixed_rank_and_options(G):
    """Fixed-rank mode (tol < 0 with k_max), plain BRP (tau_b = 0) and the greedy sampler."""
    Xs = _problems(np.float64)[:6]
    for kw, okw in [(dict(tau_b=0.0), dict(tau_b=0.0)), (dict(sampler="greedy"), dict(sampler="greedy"))]:
        outs = _run(G, Xs, 1e-7, block=8, seed=1, precision="fp64", **kw)
        for p, (X, out) in enumerate(zip(Xs, outs)):
            ref = O.rbrp_id(X, tau=1e-7, b=8, seed=1, problem=p, **okw)
            _skeletons_ok(ref, out["S"], 1e-7, (kw, p))
    outs = _run(G, Xs, -1.0, block=4, seed=2, precision="fp64", k_max=10)
    for p, (X, out) in enumerate(zip(Xs, outs)):
        ref = O.rbrp_id(X, b=4, seed=2, problem=p, k=10)
        assert out["k"] == len(ref["S"]), p
        _skeletons_ok(ref, out["S"], None, p)


def test_batched_same_as_single_problem_calls(G):
    """A batch and P separate rbrp_id calls (problem id p, FP64) give the same skeletons."""
    import torch
    Xs = _problems(np.float64)[:5]
    outs = _run(G, Xs, 1e-6, block=16, seed=11, precision="fp64")
    for p, (X, out) in enumerate(zip(Xs, outs)):
        one = G.rbrp_id(torch.from_numpy(X).to("cuda:0"), 1e-6, block=16, seed=11, problem=p, precision="fp64")
        assert one["S"].cpu().numpy().tolist() == out["S"].tolist(), p


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_shards_with_problem_base_match_one_call(G, precision):
    """Contiguous shards, each called with problem = its first index, reproduce one call."""
    from paper_2309_16002_gb300 import shard
    Xs = _problems(np.float64 if precision == "fp64" else np.float32)
    whole = _run(G, Xs, 1e-6, block=8, seed=5, precision=precision)
    for lo, hi in shard.shard_bounds([shard.problem_cost(*X.shape) for X in Xs], 3):
        if lo == hi:
            continue
        part = _run(G, Xs[lo:hi], 1e-6, block=8, seed=5, precision=precision, problem=lo)
        for j, out in enumerate(part):
            ref = whole[lo + j]
            assert out["S"].tolist() == ref["S"].tolist(), (lo + j)
            assert out["k"] == ref["k"] and out["rel_err_sq"] == ref["rel_err_sq"], (lo + j)
            assert np.array_equal(out["W"], ref["W"]), (lo + j)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_schedules_graph_and_autotune_agree(G, precision):
    """Every kernel schedule, a CUDA-graph replay and the autotuned schedule give the one-shot results."""
    import torch
    dt = np.float64 if precision == "fp64" else np.float32
    Xs = [torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0") for X in _problems(dt)]
    ref = G.rbrp_id_batched(Xs, 1e-6, block=8, seed=9, precision=precision)

    def same(outs):
        for p, (o, r) in enumerate(zip(outs, ref)):
            assert o["k"] == r["k"] and o["status"] == r["status"], p
            assert o["rel_err_sq"] == r["rel_err_sq"], p
            assert torch.equal(o["S"], r["S"]) and torch.equal(o["W"], r["W"]), p

    B = G.Batch(Xs, block=8, seed=9, precision=precision)
    tried = 0
    for threads in (256, 512):
        for per_sm in (1, 2):
            try:
                B.set_schedule(threads, per_sm)
            except G.RBRPError:
                continue  # does not fit (FP64 at two CTAs per SM)
            tried += 1
            assert B.schedule()["threads"] == threads and B.schedule()["ctas_per_sm"] == per_sm
            B.k_out.fill_(-1)
            B.run(1e-6)
            torch.cuda.synchronize()
            same(B.results())
    assert tried >= 2
    with pytest.raises(G.RBRPError):
        B.set_schedule(384, 1)
    g = B.graph(1e-6)
    B.k_out.fill_(-1)
    B.err.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    same(B.results())
    info = B.tune(1e-6, reps=1)
    assert info["threads"] in (256, 512) and info["ctas_per_sm"] in (1, 2) and info["ms"] > 0
    same(B.results())
    # a new batch of the same shape starts from the tuned schedule
    B2 = G.Batch(Xs, block=8, seed=9, precision=precision)
    assert B2.schedule()["threads"] == info["threads"] and B2.schedule()["ctas_per_sm"] == info["ctas_per_sm"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_buckets_and_row_widths_agree(G, precision):
    """The per-shape buckets (n > 128, then n <= 128) and every row width a bucket can take give
    the one-shot results bit for bit; a row width narrower than a bucket's rows is refused."""
    import torch
    dt = np.float64 if precision == "fp64" else np.float32
    Xs = [torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0") for X in _problems(dt)]
    ref = G.rbrp_id_batched(Xs, 1e-6, block=8, seed=9, precision=precision)
    B = G.Batch(Xs, block=8, seed=9, precision=precision)
    bk = B.buckets()
    assert len(bk) == 2
    assert sum(b["problems"] for b in bk) == len(Xs)
    assert bk[0]["n_max"] > 128 and bk[1]["n_max"] <= 128
    assert bk[0]["vec"] == 8 and bk[1]["vec"] == 4  # the narrowest width that holds the rows
    with pytest.raises(G.RBRPError):
        B.set_bucket_schedule(0, 256, 1, 4)  # the wide bucket's rows do not fit 4 values a lane
    with pytest.raises(G.RBRPError):
        B.set_bucket_schedule(2, 256, 1, 8)  # no such bucket
    for vec in (8, 4):
        for threads in (256, 512):
            B.set_bucket_schedule(1, threads, 1, vec)
            assert B.buckets()[1]["vec"] == vec and B.buckets()[1]["threads"] == threads
            B.k_out.fill_(-1)
            B.run(1e-6)
            torch.cuda.synchronize()
            for p, (o, r) in enumerate(zip(B.results(), ref)):
                assert o["k"] == r["k"] and o["rel_err_sq"] == r["rel_err_sq"], (vec, threads, p)
                assert torch.equal(o["S"], r["S"]) and torch.equal(o["W"], r["W"]), (vec, threads, p)
    info = B.tune(1e-6, reps=1)
    assert len(info["buckets"]) == 2 and info["ms"] > 0
    assert info["buckets"][1]["vec"] in (4, 8) and info["buckets"][0]["vec"] == 8


@pytest.mark.parametrize("sampler", ["random_exact", "greedy_exact", "greedy"])
def test_batched_exact_sampler_and_tie_fallback(G, sampler):
    """The full FP64 ranking (forced, or reached when 2000 tied greedy keys overflow the
    candidate list) draws the oracle's skeletons (FP64, problem by problem)."""
    rng = np.random.default_rng(13)
    ties = np.zeros((2000, 40))
    for i in range(2000):
        cols = rng.choice(40, size=4, replace=False)
        ties[i, cols] = rng.choice([-1.0, 1.0], size=4)
    Xs = _problems(np.float64)[:6] + [ties]
    outs = _run(G, Xs, 1e-6, block=8, seed=2, precision="fp64", sampler=sampler)
    base = sampler.replace("_exact", "")
    for p, (X, out) in enumerate(zip(Xs, outs)):
        ref = O.rbrp_id(X, tau=1e-6, b=8, seed=2, problem=p, sampler=base)
        _skeletons_ok(ref, out["S"], 1e-6, p)


def test_batched_nonfinite_and_limits(G):
    import torch
    X = np.ones((30, 6))
    X[4, 1] = np.nan
    outs = _run(G, [X, np.eye(6)], 1e-3, block=4, precision="fp64")
    assert outs[0]["status"] == 4 and outs[1]["status"] == 0 and outs[1]["k"] == 6
    with pytest.raises(G.RBRPError):
        G.rbrp_id_batched([torch.zeros((10, 300), dtype=torch.float64, device="cuda:0")], 1e-3)
    with pytest.raises(G.RBRPError):
        G.rbrp_id_batched([torch.zeros((10, 30), dtype=torch.float64, device="cuda:0")], 1e-3, block=64)


def test_batched_full_workload_sampled(G):
    """The batched benchmark's workload at full size and in its launch configuration (4096
    kernel blocks, FP32 form, tol 1e-5, b = 16, autotuned schedule, one CUDA-graph replay):
    every problem converges with W(S, :) = I, and a sample of problems meets the FP32 bar
    against the oracle run with the same Philox problem id."""
    import torch
    tol, b = 1e-5, 16
    Xs_np = WL.kernel_blocks(P=4096, seed=4)
    Xs = [torch.from_numpy(X).to("cuda:0") for X in Xs_np]
    B = G.Batch(Xs, block=b, seed=0, precision="fp32")
    B.tune(tol, reps=1)
    g = B.graph(tol)
    B.k_out.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    st = B.status.cpu().numpy()
    ks = B.k_out.cpu().numpy()
    assert (st == 0).all(), np.unique(st, return_counts=True)
    assert (ks > 0).all()
    errs = B.err.cpu().numpy()
    assert (errs <= tol).all()
    for p in range(0, 4096, 256):  # 16 problems across the size range
        X64 = Xs_np[p].astype(np.float64)
        S = B.S[p][:int(ks[p])].cpu().numpy()
        W = B.W[p][:, :int(ks[p])].cpu().numpy()
        k = len(S)
        assert np.array_equal(W[S], np.eye(k)), p
        ref = O.rbrp_id(X64, tau=tol, b=b, seed=0, problem=p)
        e_gpu = _e(X64, S, W)
        e_ref = _e(X64, ref["S"], ref["W"])
        assert P.mixed_bar(e_gpu, e_ref), (p, e_gpu, e_ref)
        e_same = float(np.sqrt(O.skeleton_error_sq(X64, S)))
        assert P.mixed_bar(e_gpu, e_same), (p, e_gpu, e_same)
        assert e_gpu ** 2 <= 1.05 * tol + 1e-10, (p, e_gpu ** 2)
        assert k <= 1.1 * len(ref["S"]) + b, (p, k, len(ref["S"]))
