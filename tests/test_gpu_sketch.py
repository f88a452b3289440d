"""GPU parity of sketchy pivoting with LUPP and the oversampled sketchy ID (Sec. 3.2, Alg. 4)
through the C ABI (rbrp_sketch_id) against the FP64 oracle (oracle/sketchy.py).

Bars:
  FP64   the LUPP pivots equal the oracle's (a mismatch only where the oracle logged a pivot
         whose |entry| was within a relative 1e-12 of the runner-up, at the first differing
         position), W within 1e-8 (relative to max |W|) of Alg. 4's, and the ID error within
         1e-10 of the oracle's.
  mixed  (FP32 sketch and LUPP; TF32 / FP32 W pass): e_gpu <= max(1.05 e_oracle,
         e_oracle + 1e-5) against the oracle's own run with the same (FP32-rounded) inputs.
W(S,:) = I in every form.
"""
import numpy as np
import pytest

from oracle import parity as P
from oracle import sketchy as K
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


def _run(G, X, Om, k, **kw):
    import torch
    out = G.rbrp_sketch_id(torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0"),
                           torch.from_numpy(np.ascontiguousarray(Om)).to("cuda:0"), k, **kw)
    torch.cuda.synchronize()
    out["S"] = out["S"].cpu().numpy()
    out["W"] = out["W"].cpu().numpy()
    return out


def _pivots_ok(ref, S):
    S_ref = ref["S"].tolist()
    S = list(S)
    if S == S_ref:
        return True, ""
    m = min(len(S), len(S_ref))
    j = next((i for i in range(m) if S[i] != S_ref[i]), m)
    gap = ref["gaps"][j] if j < len(ref["gaps"]) else np.inf
    return gap < P.NEAR_TIE, "pivots part at step %d (oracle gap %.3e)" % (j, gap)


def _fp64(G, X, Om, k, osid_cols=None, block=32):
    ref = K.sk_lupp_id(X, Om, k, osid_cols=osid_cols)
    out = _run(G, X, Om, k, precision="fp64", block=block, osid_cols=osid_cols or 0)
    ok, note = _pivots_ok(ref, out["S"])
    assert ok, note
    assert np.array_equal(out["W"][out["S"]], np.eye(len(out["S"])))
    if note:
        print("near-tie excuse: " + note)
        return ref, out
    assert np.max(np.abs(out["W"] - ref["W"])) <= 1e-8 * max(1.0, np.max(np.abs(ref["W"])))
    e_gpu = P.id_error(X, out["S"], out["W"])
    assert abs(e_gpu - np.sqrt(ref["rel_err_sq"])) <= 1e-10, (e_gpu, np.sqrt(ref["rel_err_sq"]))
    return ref, out


@pytest.mark.parametrize("n,d,k,l", [(2000, 200, 40, 120), (1037, 97, 33, 99), (777, 300, 64, 192),
                                     (4099, 128, 70, 128), (300, 50, 1, 3)])
def test_fp64_sketch_osid_matches_oracle(G, n, d, k, l):
    """Ragged row counts, k across several 32-column LUPP panels (33, 64, 70), l = 3k or capped."""
    X, _ = WL.spectral(n=n, d=d, decay="power", rate=1.0, seed=n + k)
    Om = WL.gaussian_embedding(d, l, seed=k)
    _fp64(G, X, Om, k)


def test_fp64_sketch_eq_5_2_without_oversampling(G):
    """osid_cols = k: the sketched least-squares W of Eq. (5.2); its error is above OSID's."""
    X, _ = WL.spectral(n=2000, d=200, decay="power", rate=1.0, seed=3)
    Om = WL.gaussian_embedding(200, 120, seed=4)
    ref_o, out_o = _fp64(G, X, Om, 40)
    ref_p, out_p = _fp64(G, X, Om, 40, osid_cols=40)
    assert out_o["S"].tolist() == out_p["S"].tolist()
    assert P.id_error(X, out_p["S"], out_p["W"]) >= P.id_error(X, out_o["S"], out_o["W"])


def test_fp64_sketch_gmm_full_size(G):
    """The adversarial GMM of Sec. 4 at 10^5 x 10^3 (the paper's GPU table workload), k = 100,
    l = 3k = 300: the LUPP pivots and Alg. 4's W at full size."""
    X = WL.gmm_pitfall(n=100000, d=1000, k=100, seed=6)
    Om = WL.gaussian_embedding(1000, 300, seed=100)
    ref, out = _fp64(G, X, Om, 100, block=64)
    assert len(out["S"]) == 100


def test_fp64_sketch_exact_rank_and_zero(G):
    X = WL.low_rank(n=600, d=80, r=12, seed=9)
    Om = WL.gaussian_embedding(80, 36, seed=5)
    out = _run(G, X, Om, 12, precision="fp64", block=16)
    assert len(out["S"]) == 12
    assert P.id_error(X, out["S"], out["W"]) <= 1e-12
    out = _run(G, np.zeros((50, 10)), WL.gaussian_embedding(10, 9, seed=1), 3, precision="fp64")
    assert out["k"] == 0


@pytest.mark.parametrize("prec,w_prec", [("tf32", "fp32"), ("fp32", "fp64"), ("tf32x3", "fp32")])
def test_mixed_sketch_osid_bar(G, prec, w_prec):
    X = WL.spectral(n=5000, d=300, decay="power", rate=1.0, seed=7, dtype=np.float32)[0]
    Om = WL.gaussian_embedding(300, 180, seed=8, dtype=np.float32)
    ref = K.sk_lupp_id(X, Om, 60)
    out = _run(G, X, Om, 60, precision=prec, w_precision=w_prec, block=64 if prec != "tf32x3" else 32)
    k = len(out["S"])
    assert k == 60 and len(set(out["S"].tolist())) == k
    assert np.array_equal(out["W"][out["S"]], np.eye(k))
    e_gpu = P.id_error(X, out["S"], out["W"])
    e_ref = np.sqrt(ref["rel_err_sq"])
    assert P.mixed_bar(e_gpu, e_ref), (prec, e_gpu, e_ref)


def test_sketch_argument_checks(G):
    import torch
    X = torch.zeros((64, 16), dtype=torch.float64, device="cuda:0")
    Om = torch.zeros((16, 12), dtype=torch.float64, device="cuda:0")
    with pytest.raises(G.RBRPError):
        G.rbrp_sketch_id(X, Om, 13)                      # k > l
    with pytest.raises(ValueError):
        G.rbrp_sketch_id(X, Om.float(), 4)               # FP64 sketch wants an FP64 embedding
    with pytest.raises(G.RBRPError):
        G.rbrp_sketch_id(X, Om.float(), 4, precision="tf32")  # the FP32 sketch takes FP32 X
