"""GPU test of rbrp_id_noalloc, the entry point for callers that cannot allocate device memory
(for example an engine that owns all device memory and forbids cudaMalloc): its workspace is
the library's fixed device array instead of a caller-provided buffer.

Its results must match those of rbrp_id (the allocating entry point) on the same input, for
two calls in a row, so that the second call runs on the scratch the first one left behind.
This file is collected last; it also passes when run alone in a fresh process.
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


def _e(X, S, W):
    return float(np.sqrt(O.id_error_sq(X, S, W)))


@pytest.mark.parametrize("precision,dtype,tol,b", [("fp64", np.float64, 1e-6, 16), ("tf32", np.float32, 1e-4, 32)])
def test_noalloc_matches_rbrp_id_on_two_calls(G, precision, dtype, tol, b):
    import torch
    X, _ = WL.spectral(n=2000, d=200, rate=0.9, seed=1, dtype=dtype)
    Xd = torch.from_numpy(X).to("cuda:0")
    ref = G.rbrp_id(Xd, tol, block=b, seed=0, precision=precision)
    torch.cuda.synchronize()
    S_ref = ref["S"].cpu().numpy()
    W_ref = ref["W"].cpu().numpy()
    e_ref = _e(X, S_ref, W_ref)
    kc = min(X.shape)
    skel = torch.full((kc,), -1, dtype=torch.int64, device="cuda:0")
    W = torch.full((X.shape[0], kc), np.nan, dtype=torch.float64, device="cuda:0")
    for call in range(2):
        out = G.rbrp_id_noalloc(Xd, tol, skel, W, block=b, seed=0, precision=precision)
        torch.cuda.synchronize()
        S = out["S"].cpu().numpy()
        Wk = out["W"].cpu().numpy()
        # same skeletons and, within the tolerance of the parity tests, the same ID
        assert S.tolist() == S_ref.tolist(), call
        assert abs(_e(X, S, Wk) - e_ref) <= 1e-10, call
        assert np.allclose(Wk, W_ref, rtol=1e-6, atol=1e-9), call
        assert out["k"] == ref["k"] and out["rel_err_sq"] == pytest.approx(ref["rel_err_sq"], rel=1e-12)


def test_noalloc_rejects_problems_beyond_its_scratch(G):
    import torch
    n, d = 40000, 1000  # needs far more than RBRP_NOALLOC_SCRATCH_BYTES of workspace
    opts = G.make_opts(block=64, precision="tf32")
    assert G.rbrp_workspace_size(n, d, opts) > 64 * 1024 * 1024
    X = torch.zeros((n, d), dtype=torch.float32, device="cuda:0")
    skel = torch.empty(d, dtype=torch.int64, device="cuda:0")
    W = torch.empty((n, d), dtype=torch.float64, device="cuda:0")
    with pytest.raises(G.RBRPError) as err:
        G.rbrp_id_noalloc(X, 1e-4, skel, W, block=64, precision="tf32")
    assert err.value.status == 7
