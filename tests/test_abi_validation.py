"""CPU checks of the argument validation of every C ABI entry point (include/rbrp.h).

Each case is rejected by the host-side checks that run before the first CUDA call, so no
kernel runs and no pointer is dereferenced: the buffers passed are host arrays standing in for
device buffers.  Because a regression in those checks would then hand host addresses to
kernels, the module runs only where no CUDA device is visible.
"""
import ctypes

import numpy as np
import pytest

OK, EINVAL, EWORKSPACE = 0, 1, 7


@pytest.fixture(scope="module")
def L():
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-side validation is checked where no kernel can run")
    import __graft_entry__ as g
    g.build()
    from paper_2309_16002_gb300 import rbrp
    return rbrp.load()


@pytest.fixture(scope="module")
def R():
    from paper_2309_16002_gb300 import rbrp
    return rbrp


class Bufs:
    """Host stand-ins, 256-byte aligned, large enough for a 100 x 20 problem."""

    def __init__(self, R, n=100, d=20, **kw):
        self.n, self.d = n, d
        self.o = R.make_opts(**kw)
        self.need = R.rbrp_workspace_size(n, d, self.o)
        self.raw = np.zeros(self.need + 4096, dtype=np.uint8)
        base = self.raw.ctypes.data
        self.ws = (base + 255) // 256 * 256
        self.X = np.zeros((n, d), dtype=np.float32)
        self.kc = min(n, d)
        self.skel = np.zeros(self.kc, dtype=np.int64)
        self.W = np.zeros((n, self.kc), dtype=np.float64)
        self.res = R.Result()

    def ptr(self, a):
        return ctypes.c_void_p(a.ctypes.data)


def _id(L, b, X=True, ldx=None, ldw=None, ws=None, ws_bytes=None, tol=1e-3, skel=True, W=True, res=True, o=None):
    return L.rbrp_id(b.ptr(b.X) if X else None, 0, b.n, b.d, b.d if ldx is None else ldx, tol,
                     ctypes.byref(o if o is not None else b.o), ctypes.c_void_p(b.ws if ws is None else ws),
                     b.need if ws_bytes is None else ws_bytes, b.ptr(b.skel) if skel else None,
                     b.ptr(b.W) if W else None, b.kc if ldw is None else ldw,
                     ctypes.byref(b.res) if res else None, None)


def test_rbrp_id_rejects_before_any_cuda_call(L, R):
    b = Bufs(R, block=8, precision="fp64")
    assert _id(L, b, X=False) == EINVAL
    assert _id(L, b, skel=False) == EINVAL
    assert _id(L, b, W=False) == EINVAL
    assert _id(L, b, res=False) == EINVAL
    assert _id(L, b, ldx=b.d - 1) == EINVAL                 # ldx < d
    assert _id(L, b, ldw=b.kc - 1) == EINVAL                # ldw < k_cap
    assert _id(L, b, ws=b.ws + 8) == EWORKSPACE             # misaligned workspace
    assert _id(L, b, ws_bytes=b.need - 1) == EWORKSPACE     # too small
    assert _id(L, b, tol=1.0) == EINVAL                     # tol must be < 1
    assert _id(L, b, tol=float("nan")) == EINVAL
    bad = R.make_opts(block=0, precision="fp64")
    assert _id(L, b, o=bad) == EINVAL


@pytest.mark.parametrize("field,value", [("sampler", 4), ("sampler", -1), ("w_precision", 2), ("form", 2),
                                         ("tau_b", 1.5), ("precision", 4), ("precision", -1),
                                         ("block", 257)])
def test_options_out_of_range(L, R, field, value):
    o = R.make_opts(precision="fp64")
    setattr(o, field, value)
    out = ctypes.c_size_t(0)
    assert L.rbrp_workspace_size(100, 20, ctypes.byref(o), ctypes.byref(out)) == EINVAL


def test_sizes_out_of_range(L, R):
    o = R.make_opts(precision="fp64")
    out = ctypes.c_size_t(0)
    assert L.rbrp_workspace_size(1 << 31, 20, ctypes.byref(o), ctypes.byref(out)) == EINVAL
    assert L.rbrp_workspace_size(100, 1 << 31, ctypes.byref(o), ctypes.byref(out)) == EINVAL
    assert L.rbrp_workspace_size(100, 0, ctypes.byref(o), ctypes.byref(out)) == EINVAL
    # shapes whose byte counts would overflow 64 bits are refused, not wrapped
    assert L.rbrp_workspace_size(1 << 30, 1 << 30, ctypes.byref(o), ctypes.byref(out)) == EINVAL
    assert L.rbrp_workspace_size((1 << 31) - 1, (1 << 31) - 1, ctypes.byref(o), ctypes.byref(out)) == EINVAL
    assert L.rbrp_workspace_size((1 << 31) - 1, 4096, ctypes.byref(o), ctypes.byref(out)) == OK
    assert out.value > ((1 << 31) - 1) * 4096 * 8
    assert L.rbrp_workspace_size(100, 20, ctypes.byref(o), None) == EINVAL


def test_rbrp_id_host_rejects_before_any_cuda_call(L, R):
    b = Bufs(R, block=8, precision="fp64")
    need = R.rbrp_host_workspace_size(b.n, b.d, 0, b.o)
    raw = np.zeros(need + 4096, dtype=np.uint8)
    ws = (raw.ctypes.data + 255) // 256 * 256

    def call(X=True, ws_=ws, nbytes=need, skel=True, W=True, res=True):
        return L.rbrp_id_host(b.ptr(b.X) if X else None, 0, b.n, b.d, 1e-3, ctypes.byref(b.o), ctypes.c_void_p(ws_),
                              nbytes, b.ptr(b.skel) if skel else None, b.ptr(b.W) if W else None,
                              ctypes.byref(b.res) if res else None, None)

    assert call(X=False) == EINVAL
    assert call(skel=False) == EINVAL
    assert call(W=False) == EINVAL
    assert call(res=False) == EINVAL
    assert call(ws_=0) == EINVAL
    assert call(ws_=ws + 16) == EWORKSPACE
    assert call(nbytes=need - 1) == EWORKSPACE


def test_rbrp_id_noalloc_limits(L, R):
    b = Bufs(R, block=8, precision="fp64")
    o = R.make_opts(block=8, precision="fp64")
    res = R.Result()
    # a problem whose workspace exceeds the fixed scratch is refused before the scratch is touched
    big = L.rbrp_id_noalloc(b.ptr(b.X), 0, 100000, 1000, 1000, 1e-3, ctypes.byref(o), b.ptr(b.skel), b.ptr(b.W),
                            1000, ctypes.byref(res), None)
    assert big == EWORKSPACE
    bad = R.make_opts(block=0, precision="fp64")
    assert L.rbrp_id_noalloc(b.ptr(b.X), 0, 100, 20, 20, 1e-3, ctypes.byref(bad), b.ptr(b.skel), b.ptr(b.W), 20,
                             ctypes.byref(res), None) == EINVAL


def test_batch_entry_points_reject_bad_handles_and_lists(L, R):
    assert L.rbrp_batch_run(None, 1e-3, None) == EINVAL
    f = ctypes.c_float(0)
    assert L.rbrp_batch_autotune(None, 1e-3, 1, None, ctypes.byref(f)) == EINVAL
    assert L.rbrp_batch_set_schedule(None, 256, 1) == EINVAL
    t = ctypes.c_int32(0)
    assert L.rbrp_batch_get_schedule(None, ctypes.byref(t), ctypes.byref(t), ctypes.byref(t)) == EINVAL
    L.rbrp_batch_destroy(None)                                    # no-op
    assert L.rbrp_profile_end(None) == EINVAL

    P = 2
    m = (ctypes.c_int64 * P)(100, 60)
    n = (ctypes.c_int64 * P)(20, 30)
    o = R.make_opts(block=8, precision="fp32")
    need = ctypes.c_size_t(0)
    assert L.rbrp_batched_workspace_size(P, m, n, ctypes.byref(o), ctypes.byref(need)) == OK
    raw = np.zeros(need.value + 4096, dtype=np.uint8)
    ws = (raw.ctypes.data + 255) // 256 * 256
    X = [np.zeros((100, 20), np.float32), np.zeros((60, 30), np.float32)]
    S = [np.zeros(20, np.int64), np.zeros(30, np.int64)]
    W = [np.zeros((100, 20)), np.zeros((60, 30))]
    k_out = np.zeros(P, np.int64)
    err = np.zeros(P)
    st = np.zeros(P, np.int32)

    def arr(xs, null_at=None):
        return (ctypes.c_void_p * P)(*[None if i == null_at else x.ctypes.data for i, x in enumerate(xs)])

    def create(Xa=None, Sa=None, Wa=None, ws_=ws, nbytes=None, out=True, P_=P):
        h = ctypes.c_void_p(None)
        rc = L.rbrp_batch_create(P_, Xa if Xa is not None else arr(X), m, n, 0, ctypes.byref(o), ctypes.c_void_p(ws_),
                                 need.value if nbytes is None else nbytes, Sa if Sa is not None else arr(S),
                                 Wa if Wa is not None else arr(W), k_out.ctypes.data, err.ctypes.data,
                                 st.ctypes.data, None, ctypes.byref(h) if out else None)
        assert not h.value  # no handle is returned on any rejected call
        return rc

    assert create(out=False) == EINVAL
    assert create(P_=0) == EINVAL
    assert create(Xa=arr(X, null_at=1)) == EINVAL
    assert create(Sa=arr(S, null_at=0)) == EINVAL
    assert create(Wa=arr(W, null_at=1)) == EINVAL
    assert create(ws_=ws + 64) == EWORKSPACE
    assert create(nbytes=need.value - 1) == EWORKSPACE

    # the one-shot form: P = 0 is valid and does nothing; tol >= 1 is refused
    assert L.rbrp_id_batched(0, None, None, None, 0, 1e-3, ctypes.byref(o), None, 0, None, None, None, None, None,
                             None) == OK
    assert L.rbrp_id_batched(P, arr(X), m, n, 0, 1.0, ctypes.byref(o), ctypes.c_void_p(ws), need.value, arr(S),
                             arr(W), k_out.ctypes.data, err.ctypes.data, st.ctypes.data, None) == EINVAL
