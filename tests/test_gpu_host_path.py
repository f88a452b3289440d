"""GPU checks of rbrp_id_host (host buffers in and out) against rbrp_id on device buffers.

The host entry point copies X in, runs the same device path, and copies W out by
row ranges on a second stream while the later ranges of the W solve (Alg. 3)
are still running.  The skeletons must be identical and W bit-identical to the
device call (same kernels on the same rows), including rows on both sides of a
range boundary and the identity rows W(S, :) = I; the error is checked against
the FP64 oracle's recomputation.
"""
import numpy as np
import pytest

from oracle import rbrp as O
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


def _both(G, X, tol, **kw):
    import torch
    dev = G.rbrp_id(torch.from_numpy(X).to("cuda:0"), tol, **kw)
    torch.cuda.synchronize()
    d = dict(k=dev["k"], S=dev["S"].cpu().numpy(), W=dev["W"].cpu().numpy(), rel=dev["rel_err_sq"],
             converged=dev["converged"])
    skel_h = torch.empty(G.k_cap(*X.shape, kw.get("k_max", 0)), dtype=torch.int64).pin_memory()
    W_h = torch.empty((X.shape[0], skel_h.numel()), dtype=torch.float64).pin_memory()
    host = G.rbrp_id_host(X, tol, skel_out=skel_h, W_out=W_h, **kw)
    h = dict(k=host["k"], S=host["S"].numpy().copy(), W=host["W"].numpy().copy(), rel=host["rel_err_sq"],
             converged=host["converged"])
    return d, h


@pytest.mark.parametrize("n", [50000, 19456 * 2 + 128 * 3 + 77])
def test_host_path_tf32_fp32w_matches_device(G, n):
    """TF32 chain with the tensor-core FP32 W solve: several row ranges of one tile per SM
    (19456 rows on 152 SMs), the last one ragged."""
    X = WL.zipf_gmm(n=n, d=160, clusters=24, seed=11)
    d, h = _both(G, X, 1e-3, block=32, precision="tf32", w_precision="fp32", seed=5)
    assert h["k"] == d["k"] > 0
    assert np.array_equal(h["S"], d["S"])
    assert h["rel"] == d["rel"]
    assert np.array_equal(h["W"], d["W"]), np.argwhere(h["W"] != d["W"])[:5]
    assert np.array_equal(h["W"][h["S"]], np.eye(h["k"]))
    e2 = O.id_error_sq(X.astype(np.float64), h["S"], h["W"])
    assert e2 <= 1.05 * 1e-3, e2


def test_host_path_fp64_matches_device(G):
    """FP64 chain and FP64 W (one range, handed over after the whole solve)."""
    X, _ = WL.spectral(n=3000, d=120, rate=0.85, seed=3)
    d, h = _both(G, X, 1e-8, block=16, precision="fp64", seed=2)
    assert h["k"] == d["k"] > 0
    assert np.array_equal(h["S"], d["S"])
    assert np.array_equal(h["W"], d["W"])
    assert np.array_equal(h["W"][h["S"]], np.eye(h["k"]))


def test_host_path_fixed_rank_not_converged(G):
    """k_max reached first (status not converged): W still arrives for the k_max columns."""
    X = WL.zipf_gmm(n=30000, d=96, clusters=40, seed=12)
    d, h = _both(G, X, 1e-9, block=16, precision="tf32", w_precision="fp32", seed=1, k_max=48)
    assert h["k"] == d["k"] == 48
    assert not h["converged"] and not d["converged"]
    assert np.array_equal(h["S"], d["S"])
    assert np.array_equal(h["W"], d["W"])
