"""Failure detection on the GPU without a fault: the bounded device waits give up.

Every wait of the library's kernels on another part of the same launch is bounded (the
mbarrier waits of the tensor-core update, the grid barriers of the cooperative sampler).
Setting the poll limit to 1 makes a healthy run's waits give up; the call must then
return RBRP_ETIMEOUT (not hang, not fault), and a normal call on the same workspace
afterwards must still give the oracle's result.  No test here faults, traps or hangs a GPU.
"""
import numpy as np
import pytest

from oracle import rbrp as O
from paper_2309_16002_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

RBRP_ETIMEOUT = 6


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2309_16002_gb300 import rbrp
    rbrp.load()
    yield rbrp
    rbrp.set_wait_limits(0, 0)


def _timed_out(G, Xd, tol, ws, **kw):
    with pytest.raises(G.RBRPError) as e:
        G.rbrp_id(Xd, tol, workspace=ws, **kw)
    return e.value.status


@pytest.mark.parametrize("precision", ["tf32", "tf32x3"])
def test_update_mbarrier_wait_gives_up_and_workspace_recovers(G, precision):
    """Persistent tensor-core update (TF32 or its 3xTF32 split, b = 64): its first wait on a
    TMA load (or, split, on the converter warps) cannot be met within one poll, so the CTA
    aborts, drains its own copies and MMAs, frees its tensor memory and reports RBRP_ETIMEOUT;
    the next call on the same workspace is exact again."""
    import torch
    X, _ = WL.spectral(n=6000, d=300, rate=0.93, seed=31, dtype=np.float32)
    Xd = torch.from_numpy(X).to("cuda:0")
    kw = dict(block=64, seed=2, precision=precision)
    ws = G.Workspace(*X.shape, G.make_opts(**kw), Xd.device)
    try:
        G.set_wait_limits(1, 0)
        assert _timed_out(G, Xd, 1e-4, ws, **kw) == RBRP_ETIMEOUT
    finally:
        G.set_wait_limits(0, 0)
    torch.cuda.synchronize()
    out = G.rbrp_id(Xd, 1e-4, workspace=ws, **kw)
    ref = O.rbrp_id(X, tau=1e-4, b=64, seed=2)
    S = out["S"].cpu().numpy()
    W = out["W"].cpu().numpy()
    e_gpu = np.sqrt(O.id_error_sq(X, S, W))
    e_ref = np.sqrt(O.id_error_sq(X, ref["S"], ref["W"]))
    assert e_gpu <= max(1.05 * e_ref, e_ref + 1e-5), (e_gpu, e_ref)
    assert np.array_equal(W[S], np.eye(len(S)))


def test_sampler_grid_barrier_gives_up_and_workspace_recovers(G):
    """Cooperative sampler (FP64 path): with one poll per grid barrier some CTA gives up,
    the call reports RBRP_ETIMEOUT, and the next call reproduces the oracle's skeletons."""
    import torch
    X, _ = WL.spectral(n=120000, d=48, rate=0.9, seed=32)
    Xd = torch.from_numpy(X).to("cuda:0")
    kw = dict(block=16, seed=5, precision="fp64")
    ws = G.Workspace(*X.shape, G.make_opts(**kw), Xd.device)
    try:
        G.set_wait_limits(0, 1)
        assert _timed_out(G, Xd, 1e-6, ws, **kw) == RBRP_ETIMEOUT
    finally:
        G.set_wait_limits(0, 0)
    torch.cuda.synchronize()
    out = G.rbrp_id(Xd, 1e-6, workspace=ws, **kw)
    ref = O.rbrp_id(X, tau=1e-6, b=16, seed=5)
    assert out["S"].cpu().numpy().tolist() == ref["S"].tolist()
