"""The device-side block loop (a CUDA graph whose while node repeats one block of Alg. 2,
its condition set by the stopping test on the device) against the host-queued loop: the
same kernels, so identical skeletons, W and residuals, bit for bit; the graph built by the
first call with a set of buffers is reused by later calls (any tolerance)."""
import numpy as np
import pytest

from oracle import parity as P
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
    yield rbrp
    rbrp.set_loop_mode("device")


def _both(G, X, tol, **kw):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0")
    ws = G.Workspace(*X.shape, G.make_opts(**{k: v for k, v in kw.items() if k in (
        "block", "precision", "k_max", "seed", "w_precision", "chain")}), Xd.device)
    outs = {}
    for mode in ("host", "device", "device"):  # the second device call reuses the graph
        G.set_loop_mode(mode)
        o = G.rbrp_id(Xd, tol, workspace=ws, **kw)
        torch.cuda.synchronize()
        outs.setdefault(mode, []).append({"S": o["S"].cpu().numpy().copy(), "W": o["W"].cpu().numpy().copy(),
                                          "k": o["k"], "blocks": o["blocks"], "rel": o["rel_err_sq"]})
    G.set_loop_mode("device")
    h = outs["host"][0]
    for dv in outs["device"]:
        assert dv["k"] == h["k"] and dv["blocks"] == h["blocks"]
        assert np.array_equal(dv["S"], h["S"]) and np.array_equal(dv["W"], h["W"])
        assert dv["rel"] == h["rel"]
    return h


@pytest.mark.parametrize("prec,chain", [("fp64", "default"), ("tf32", "default"), ("tf32", "fp64"),
                                        ("tf32x3", "default")])
def test_device_loop_matches_host_loop(G, prec, chain):
    X, _ = WL.spectral(n=3000, d=150, rate=0.9, seed=41, dtype=np.float64 if prec == "fp64" else np.float32)
    h = _both(G, X, 1e-6 if prec == "fp64" else 1e-4, block=16, seed=3, precision=prec, chain=chain)
    if prec == "fp64":
        ref = O.rbrp_id(X, tau=1e-6, b=16, seed=3)
        ok, note = P.fp64_skeleton_check(ref, h["S"], 1e-6)
        assert ok, note


def test_device_loop_fixed_rank_zero_and_one_block(G):
    X, _ = WL.spectral(n=800, d=60, rate=0.85, seed=42)
    h = _both(G, X, -1.0, block=8, seed=1, precision="fp64", k_max=23)
    assert h["k"] == 23
    h = _both(G, np.zeros((40, 8)), 1e-3, block=4, precision="fp64")
    assert h["k"] == 0
    h = _both(G, X, -1.0, block=16, seed=2, precision="fp64", k_max=16)
    assert h["k"] == 16 and h["blocks"] >= 1  # the robust filter may accept fewer than b per block


def test_device_loop_graph_serves_any_tolerance(G):
    """One workspace, one graph, three tolerances: each call matches a host-loop call."""
    import torch
    X = WL.zipf_gmm(n=8000, d=200, clusters=20, seed=3)
    Xd = torch.from_numpy(X).to("cuda:0")
    ws = G.Workspace(*X.shape, G.make_opts(block=32, precision="tf32"), Xd.device)
    for tol in (1e-2, 1e-3, 1e-4):
        res = {}
        for mode in ("device", "host"):
            G.set_loop_mode(mode)
            o = G.rbrp_id(Xd, tol, workspace=ws, block=32, precision="tf32")
            torch.cuda.synchronize()
            res[mode] = (o["S"].cpu().numpy().copy(), o["rel_err_sq"])
        G.set_loop_mode("device")
        assert np.array_equal(res["device"][0], res["host"][0]) and res["device"][1] == res["host"][1]
        assert res["device"][1] <= tol
