"""Thin ctypes binding of librbrp.so (include/rbrp.h).

Argument marshalling only: every step of RBRP runs in the CUDA library.  PyTorch
supplies device memory (the workspace and the outputs) and the current stream.
There is no CPU fallback: if the library is missing, loading it raises.

Functions mirror the C ABI:
  rbrp_id(X, tol, ...)          X a CUDA tensor (FP32 or FP64, row-major)
  rbrp_id_host(X, tol, ...)     X a host tensor/array; copies inside the call
  rbrp_workspace_size(n, d, opts), rbrp_host_workspace_size(n, d, x_is_fp64, opts)
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "librbrp.so")
_lib = None

PRECISIONS = {"fp64": 0, "tf32": 1, "fp32": 2, "tf32x3": 3}
SAMPLERS = {"random": 0, "greedy": 1, "random_exact": 2, "greedy_exact": 3}
W_PRECISIONS = {"fp64": 0, "fp32": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "non-finite value",
          5: "not converged", 6: "timeout", 7: "workspace"}
RBRP_ENOTCONVERGED = 5

EXPORTS = ["rbrp_default_opts", "rbrp_workspace_size", "rbrp_id", "rbrp_host_workspace_size", "rbrp_id_host",
           "rbrp_status_string", "rbrp_last_cuda_error", "rbrp_profile_begin", "rbrp_profile_end",
           "rbrp_id_noalloc", "rbrp_batched_workspace_size", "rbrp_id_batched", "rbrp_batch_create",
           "rbrp_batch_run", "rbrp_batch_autotune", "rbrp_batch_set_schedule", "rbrp_batch_get_schedule",
           "rbrp_batch_buckets", "rbrp_batch_get_bucket", "rbrp_batch_set_bucket_schedule", "rbrp_batch_destroy", "rbrp_set_wait_limits", "rbrp_sketch_workspace_size", "rbrp_sketch_id",
           "rbrp_set_loop_mode", "rbrp_shard_workspace_size", "rbrp_shard_create", "rbrp_shard_draw",
           "rbrp_shard_rows", "rbrp_shard_block", "rbrp_shard_l_rows", "rbrp_shard_w", "rbrp_shard_destroy"]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("block", ctypes.c_int32), ("tau_b", ctypes.c_double),
                ("k_max", ctypes.c_int64), ("seed", ctypes.c_uint64), ("problem", ctypes.c_uint64),
                ("sampler", ctypes.c_int32), ("w_precision", ctypes.c_int32), ("form", ctypes.c_int32),
                ("chain", ctypes.c_int32)]


class SketchOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("block", ctypes.c_int32), ("w_precision", ctypes.c_int32),
                ("osid_cols", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("blocks", ctypes.c_int64), ("d0", ctypes.c_double),
                ("d_final", ctypes.c_double), ("rel_err_sq", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("update_launches", ctypes.c_int64), ("update_ms", ctypes.c_double),
                ("wsolve_calls", ctypes.c_int64), ("wsolve_ms", ctypes.c_double), ("blocks", ctypes.c_int64),
                ("skeletons", ctypes.c_int64)]


class RBRPError(RuntimeError):
    def __init__(self, status, where, cuda_err=0):
        self.status = status
        msg = "%s: %s" % (where, STATUS.get(status, str(status)))
        if status == 3:
            msg += " (cudaError %d)" % cuda_err
        super().__init__(msg)


def lib_path():
    return _LIBPATH


def load():
    """Load librbrp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise RuntimeError("librbrp.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(_LIBPATH)
    vp, sz, i64, dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_double
    L.rbrp_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.rbrp_default_opts.restype = None
    L.rbrp_workspace_size.argtypes = [i64, i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    L.rbrp_workspace_size.restype = ctypes.c_int
    L.rbrp_host_workspace_size.argtypes = [i64, i64, ctypes.c_int, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    L.rbrp_host_workspace_size.restype = ctypes.c_int
    L.rbrp_id.argtypes = [vp, ctypes.c_int, i64, i64, i64, dbl, ctypes.POINTER(Opts), vp, sz, vp, vp, i64,
                          ctypes.POINTER(Result), vp]
    L.rbrp_id.restype = ctypes.c_int
    L.rbrp_id_host.argtypes = [vp, ctypes.c_int, i64, i64, dbl, ctypes.POINTER(Opts), vp, sz, vp, vp,
                               ctypes.POINTER(Result), vp]
    L.rbrp_id_host.restype = ctypes.c_int
    L.rbrp_status_string.argtypes = [ctypes.c_int]
    L.rbrp_status_string.restype = ctypes.c_char_p
    L.rbrp_last_cuda_error.argtypes = []
    L.rbrp_last_cuda_error.restype = ctypes.c_int
    L.rbrp_id_noalloc.argtypes = [vp, ctypes.c_int, i64, i64, i64, dbl, ctypes.POINTER(Opts), vp, vp, i64,
                                  ctypes.POINTER(Result), vp]
    L.rbrp_id_noalloc.restype = ctypes.c_int
    P64 = ctypes.POINTER(ctypes.c_int64)
    L.rbrp_batched_workspace_size.argtypes = [ctypes.c_int32, P64, P64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    L.rbrp_batched_workspace_size.restype = ctypes.c_int
    L.rbrp_id_batched.argtypes = [ctypes.c_int32, ctypes.POINTER(vp), P64, P64, ctypes.c_int, dbl,
                                  ctypes.POINTER(Opts), vp, sz, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp,
                                  vp]
    L.rbrp_id_batched.restype = ctypes.c_int
    L.rbrp_batch_create.argtypes = [ctypes.c_int32, ctypes.POINTER(vp), P64, P64, ctypes.c_int, ctypes.POINTER(Opts),
                                    vp, sz, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp, vp,
                                    ctypes.POINTER(vp)]
    L.rbrp_batch_create.restype = ctypes.c_int
    L.rbrp_batch_run.argtypes = [vp, dbl, vp]
    L.rbrp_batch_run.restype = ctypes.c_int
    L.rbrp_batch_autotune.argtypes = [vp, dbl, ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_float)]
    L.rbrp_batch_autotune.restype = ctypes.c_int
    L.rbrp_batch_set_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    L.rbrp_batch_set_schedule.restype = ctypes.c_int
    P32 = ctypes.POINTER(ctypes.c_int32)
    L.rbrp_batch_get_schedule.argtypes = [vp, P32, P32, P32]
    L.rbrp_batch_get_schedule.restype = ctypes.c_int
    L.rbrp_batch_buckets.argtypes = [vp]
    L.rbrp_batch_buckets.restype = ctypes.c_int32
    L.rbrp_batch_get_bucket.argtypes = [vp, ctypes.c_int32, P32, ctypes.POINTER(ctypes.c_int64), P32, P32, P32, P32]
    L.rbrp_batch_get_bucket.restype = ctypes.c_int
    L.rbrp_batch_set_bucket_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.rbrp_batch_set_bucket_schedule.restype = ctypes.c_int
    L.rbrp_batch_destroy.argtypes = [vp]
    L.rbrp_batch_destroy.restype = None
    L.rbrp_sketch_workspace_size.argtypes = [i64, i64, i64, i64, ctypes.POINTER(SketchOpts), ctypes.POINTER(sz)]
    L.rbrp_sketch_workspace_size.restype = ctypes.c_int
    L.rbrp_sketch_id.argtypes = [vp, ctypes.c_int, i64, i64, i64, vp, i64, i64, ctypes.POINTER(SketchOpts), vp, sz,
                                 vp, vp, i64, ctypes.POINTER(Result), vp]
    L.rbrp_sketch_id.restype = ctypes.c_int
    PD = ctypes.POINTER(ctypes.c_double)
    L.rbrp_shard_workspace_size.argtypes = [i64, i64, i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    L.rbrp_shard_workspace_size.restype = ctypes.c_int
    L.rbrp_shard_create.argtypes = [vp, ctypes.c_int, i64, i64, i64, i64, i64, ctypes.POINTER(Opts), vp, sz, vp,
                                    ctypes.POINTER(vp), PD]
    L.rbrp_shard_create.restype = ctypes.c_int
    L.rbrp_shard_draw.argtypes = [vp, P64, PD, P64]
    L.rbrp_shard_draw.restype = ctypes.c_int
    L.rbrp_shard_rows.argtypes = [vp, P64, i64, PD, P32]
    L.rbrp_shard_rows.restype = ctypes.c_int
    L.rbrp_shard_block.argtypes = [vp, PD, P64, i64, P64, P64, PD]
    L.rbrp_shard_block.restype = ctypes.c_int
    L.rbrp_shard_l_rows.argtypes = [vp, P64, i64, i64, PD, P32]
    L.rbrp_shard_l_rows.restype = ctypes.c_int
    L.rbrp_shard_w.argtypes = [vp, PD, P64, i64, vp, i64]
    L.rbrp_shard_w.restype = ctypes.c_int
    L.rbrp_shard_destroy.argtypes = [vp]
    L.rbrp_shard_destroy.restype = None
    L.rbrp_set_loop_mode.argtypes = [ctypes.c_int32]
    L.rbrp_set_loop_mode.restype = ctypes.c_int
    L.rbrp_set_wait_limits.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    L.rbrp_set_wait_limits.restype = None
    L.rbrp_profile_begin.argtypes = []
    L.rbrp_profile_begin.restype = None
    L.rbrp_profile_end.argtypes = [ctypes.POINTER(Profile)]
    L.rbrp_profile_end.restype = ctypes.c_int
    _lib = L
    return L


LOOP_MODES = {"device": 0, "host": 1}


def set_loop_mode(mode="device"):
    """How later calls drive the blocks of Alg. 2: "device" (a CUDA graph's while node) or "host"."""
    st = load().rbrp_set_loop_mode(LOOP_MODES[mode])
    if st != 0:
        raise RBRPError(st, "rbrp_set_loop_mode")


def set_wait_limits(mbarrier_polls=0, barrier_polls=0):
    """Poll limits of the library's bounded device waits for later calls (0: the default)."""
    load().rbrp_set_wait_limits(int(mbarrier_polls), int(barrier_polls))


def rbrp_profile_begin():
    load().rbrp_profile_begin()


def rbrp_profile_end():
    p = Profile()
    st = load().rbrp_profile_end(ctypes.byref(p))
    if st != 0:
        raise RBRPError(st, "rbrp_profile_end", load().rbrp_last_cuda_error())
    return {f: getattr(p, f) for f, _ in Profile._fields_}


FORMS = {"residual": 0, "downdate": 1}
CHAINS = {"default": 0, "fp64": 1}


def make_opts(block=64, precision="tf32", tau_b=-1.0, k_max=0, seed=0, problem=0, sampler="random",
              w_precision="fp64", form="residual", chain="default"):
    o = Opts()
    load().rbrp_default_opts(ctypes.byref(o))
    o.precision = PRECISIONS[precision]
    o.block = int(block)
    o.tau_b = float(tau_b)
    o.k_max = int(k_max)
    o.seed = int(seed)
    o.problem = int(problem)
    o.sampler = SAMPLERS[sampler]
    o.w_precision = W_PRECISIONS[w_precision]
    o.form = FORMS[form]
    o.chain = CHAINS[chain]
    return o


def k_cap(n, d, k_max=0):
    kc = min(n, d)
    return min(kc, k_max) if k_max and k_max > 0 else kc


def rbrp_workspace_size(n, d, opts):
    out = ctypes.c_size_t(0)
    st = load().rbrp_workspace_size(int(n), int(d), ctypes.byref(opts), ctypes.byref(out))
    if st != 0:
        raise RBRPError(st, "rbrp_workspace_size")
    return out.value


def rbrp_host_workspace_size(n, d, x_is_fp64, opts):
    out = ctypes.c_size_t(0)
    st = load().rbrp_host_workspace_size(int(n), int(d), int(x_is_fp64), ctypes.byref(opts), ctypes.byref(out))
    if st != 0:
        raise RBRPError(st, "rbrp_host_workspace_size")
    return out.value


def _check(status, where, allow_notconverged=True):
    if status == 0 or (allow_notconverged and status == RBRP_ENOTCONVERGED):
        return
    raise RBRPError(status, where, load().rbrp_last_cuda_error())


def _result_dict(res, status):
    return dict(k=int(res.k), blocks=int(res.blocks), d0=res.d0, d_final=res.d_final, rel_err_sq=res.rel_err_sq,
                converged=(status == 0))


# The C ABI receives plain pointers and sizes, so the binding checks every buffer it
# passes (dtype, device, shape, layout) before the call: a wrong one would otherwise
# be read or written out of bounds.
def _check_x(X, cuda):
    import torch
    if X.dim() != 2 or X.stride(1) != 1 or X.is_cuda != cuda:
        raise ValueError("X must be a 2-D %s tensor with unit column stride" % ("CUDA" if cuda else "host"))
    if X.dtype not in (torch.float32, torch.float64):
        raise ValueError("X must be float32 or float64")
    if X.shape[0] < 1 or X.shape[1] < 1:
        raise ValueError("X must have at least one row and one column")


def _check_outputs(skel, W, n, kc, device=None, exact_host_shape=False):
    """skel: int64[>= kc]; W: FP64 n x (>= kc) rows with unit column stride, row stride >= kc
    (host outputs of rbrp_id_host: exactly n x kc, C-contiguous, since the copy assumes that pitch)."""
    import torch
    cuda = device is not None
    for name, t in (("skel", skel), ("W", W)):
        if t.is_cuda != cuda or (cuda and t.device != device):
            raise ValueError("%s must be a %s tensor" % (name, "CUDA tensor on %s" % device if cuda else "host"))
    if skel.dtype != torch.int64 or not skel.is_contiguous() or skel.numel() < kc:
        raise ValueError("skel must be a contiguous int64 tensor of at least k_cap = %d entries" % kc)
    if W.dtype != torch.float64 or W.dim() != 2 or W.stride(1) != 1:
        raise ValueError("W must be a 2-D float64 tensor with unit column stride")
    if exact_host_shape:
        if tuple(W.shape) != (n, kc) or not W.is_contiguous():
            raise ValueError("W must be a C-contiguous float64 host tensor of shape (%d, %d)" % (n, kc))
    elif W.shape[0] < n or W.shape[1] < kc or W.stride(0) < kc:
        raise ValueError("W must hold n = %d rows of k_cap = %d columns" % (n, kc))


class Workspace:
    """Device buffers for repeated rbrp_id calls of one shape (allocated once by PyTorch)."""

    def __init__(self, n, d, opts, device=None):
        import torch
        self.n, self.d = int(n), int(d)
        self.opts = opts
        self.kc = k_cap(n, d, opts.k_max)
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.ws = torch.empty(rbrp_workspace_size(n, d, opts) + 256, dtype=torch.uint8, device=dev)
        self.skel = torch.empty(self.kc, dtype=torch.int64, device=dev)
        self.W = torch.empty((self.n, self.kc), dtype=torch.float64, device=dev)

    def ws_ptr(self):
        p = self.ws.data_ptr()
        return (p + 255) // 256 * 256

    def ws_bytes(self):
        return self.ws.numel() - (self.ws_ptr() - self.ws.data_ptr())


def rbrp_id(X, tol, block=64, seed=0, precision="tf32", tau_b=-1.0, k_max=0, problem=0, sampler="random",
            w_precision="fp64", workspace=None, stream=None, form="residual", chain="default"):
    """Row ID of a CUDA tensor X (n x d, FP32/FP64, row-major rows) by RBRP (Alg. 2) and Alg. 3.

    Returns dict(S (int64 CUDA tensor, acceptance order), W (n x k FP64 CUDA tensor), k, blocks,
    rel_err_sq (= ||d||_1 / ||d0||_1), d0, d_final, converged).
    """
    import torch
    _check_x(X, cuda=True)
    n, d = X.shape
    opts = make_opts(block, precision, tau_b, k_max, seed, problem, sampler, w_precision, form, chain)
    if workspace is not None and ((workspace.n, workspace.d) != (n, d) or workspace.kc < k_cap(n, d, k_max)):
        raise ValueError("workspace was made for %d x %d, k_cap %d" % (workspace.n, workspace.d, workspace.kc))
    ws = workspace if workspace is not None else Workspace(n, d, opts, X.device)
    if ws.ws.device != X.device:
        raise ValueError("workspace and X are on different devices")
    res = Result()
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    st = load().rbrp_id(ctypes.c_void_p(X.data_ptr()), int(X.dtype == torch.float64), n, d, X.stride(0), float(tol),
                        ctypes.byref(opts), ctypes.c_void_p(ws.ws_ptr()), ws.ws_bytes(),
                        ctypes.c_void_p(ws.skel.data_ptr()), ctypes.c_void_p(ws.W.data_ptr()), ws.kc,
                        ctypes.byref(res), ctypes.c_void_p(s.cuda_stream))
    _check(st, "rbrp_id")
    out = _result_dict(res, st)
    k = out["k"]
    out["S"] = ws.skel[:k]
    out["W"] = ws.W[:, :k]
    return out


def rbrp_id_noalloc(X, tol, skel_out, W_out, block=64, seed=0, precision="tf32", tau_b=-1.0, k_max=0, problem=0,
                    sampler="random", w_precision="fp64", stream=None, form="residual", chain="default"):
    """rbrp_id without any device allocation by the library: the workspace is the library's
    fixed device array (RBRP_NOALLOC_SCRATCH_BYTES).  For callers that cannot allocate; the
    outputs skel_out (int64[k_cap]) and W_out (FP64 n x k_cap) are the caller's CUDA tensors.
    The first call on a device commits the array (see include/rbrp.h): make it at start-up."""
    import torch
    _check_x(X, cuda=True)
    n, d = X.shape
    _check_outputs(skel_out, W_out, n, k_cap(n, d, k_max), device=X.device)
    opts = make_opts(block, precision, tau_b, k_max, seed, problem, sampler, w_precision, form, chain)
    res = Result()
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    st = load().rbrp_id_noalloc(ctypes.c_void_p(X.data_ptr()), int(X.dtype == torch.float64), n, d, X.stride(0),
                                float(tol), ctypes.byref(opts), ctypes.c_void_p(skel_out.data_ptr()),
                                ctypes.c_void_p(W_out.data_ptr()), W_out.stride(0), ctypes.byref(res),
                                ctypes.c_void_p(s.cuda_stream))
    _check(st, "rbrp_id_noalloc")
    out = _result_dict(res, st)
    k = out["k"]
    out["S"] = skel_out[:k]
    out["W"] = W_out[:, :k]
    return out


class HostWorkspace:
    """Device workspace for rbrp_id_host of one shape."""

    def __init__(self, n, d, x_is_fp64, opts, device=None):
        import torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.ws = torch.empty(rbrp_host_workspace_size(n, d, x_is_fp64, opts) + 256, dtype=torch.uint8, device=dev)

    def ptr(self):
        return (self.ws.data_ptr() + 255) // 256 * 256

    def nbytes(self):
        return self.ws.numel() - (self.ptr() - self.ws.data_ptr())


def rbrp_id_host(X, tol, block=64, seed=0, precision="tf32", tau_b=-1.0, k_max=0, problem=0, sampler="random",
                 w_precision="fp64", workspace=None, skel_out=None, W_out=None, stream=None, form="residual",
                 chain="default"):
    """rbrp_id on host buffers: X (numpy array or CPU tensor, C-contiguous FP32/FP64).

    skel_out / W_out: optional preallocated host outputs (int64[k_cap], FP64 n x k_cap, pinned
    tensors make the copies asynchronous).  Returns the same dict as rbrp_id with host S and W.
    """
    import torch
    Xt = torch.as_tensor(X)
    if not Xt.is_contiguous():
        raise ValueError("X must be a C-contiguous 2-D host array")
    _check_x(Xt, cuda=False)
    n, d = Xt.shape
    fp64 = int(Xt.dtype == torch.float64)
    opts = make_opts(block, precision, tau_b, k_max, seed, problem, sampler, w_precision, form, chain)
    kc = k_cap(n, d, k_max)
    skel = skel_out if skel_out is not None else torch.empty(kc, dtype=torch.int64)
    W = W_out if W_out is not None else torch.empty((n, kc), dtype=torch.float64)
    _check_outputs(skel, W, n, kc, exact_host_shape=True)
    if workspace is not None and workspace.nbytes() < rbrp_host_workspace_size(n, d, fp64, opts):
        raise ValueError("workspace too small for this problem")
    ws = workspace if workspace is not None else HostWorkspace(n, d, fp64, opts)
    res = Result()
    s = stream if stream is not None else torch.cuda.current_stream()
    st = load().rbrp_id_host(ctypes.c_void_p(Xt.data_ptr()), fp64, n, d, float(tol), ctypes.byref(opts),
                             ctypes.c_void_p(ws.ptr()), ws.nbytes(), ctypes.c_void_p(skel.data_ptr()),
                             ctypes.c_void_p(W.data_ptr()), ctypes.byref(res), ctypes.c_void_p(s.cuda_stream))
    _check(st, "rbrp_id_host")
    out = _result_dict(res, st)
    k = out["k"]
    out["S"] = skel[:k]
    out["W"] = W[:, :k]
    return out


def exported_symbols():
    """Names of the C ABI entry points the binding expects (declared in include/rbrp.h)."""
    return list(EXPORTS)


def as_numpy(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


class Batch:
    """One list of problems bound to preallocated outputs and workspace (rbrp_batch_* of include/rbrp.h).

    run(tol, stream) queues one solve of every problem (a memset and one kernel
    launch); graph(tol) captures that in a torch.cuda.CUDAGraph for replay;
    tune(tol) times the kernel schedules and keeps the fastest.
    """

    def __init__(self, Xs, block=16, seed=0, precision="fp32", tau_b=-1.0, k_max=0, sampler="random", problem=0,
                 stream=None, handle=True):
        import torch
        self.P = len(Xs)
        if self.P == 0:
            raise ValueError("empty batch")
        dt = Xs[0].dtype
        dev = Xs[0].device
        if dt not in (torch.float32, torch.float64):
            raise ValueError("Xs must be float32 or float64")
        for X in Xs:
            if not X.is_cuda or X.dim() != 2 or X.dtype != dt or not X.is_contiguous() or X.device != dev:
                raise ValueError("Xs must be contiguous 2-D CUDA tensors of one dtype on one device")
        self.Xs = Xs
        self.fp64_in = int(dt == torch.float64)
        self.opts = make_opts(block, precision, tau_b, k_max, seed, problem, sampler, "fp64")
        P = self.P
        self.m = (ctypes.c_int64 * P)(*[int(X.shape[0]) for X in Xs])
        self.n = (ctypes.c_int64 * P)(*[int(X.shape[1]) for X in Xs])
        L = load()
        need = ctypes.c_size_t(0)
        st = L.rbrp_batched_workspace_size(P, self.m, self.n, ctypes.byref(self.opts), ctypes.byref(need))
        _check(st, "rbrp_batched_workspace_size", allow_notconverged=False)
        self.need = need.value
        self.ws = torch.empty(self.need + 256, dtype=torch.uint8, device=dev)
        self.wp = (self.ws.data_ptr() + 255) // 256 * 256
        kcs = [k_cap(int(X.shape[0]), int(X.shape[1]), k_max) for X in Xs]
        self.S = [torch.empty(kc, dtype=torch.int64, device=dev) for kc in kcs]
        self.W = [torch.empty((int(X.shape[0]), kc), dtype=torch.float64, device=dev) for X, kc in zip(Xs, kcs)]
        self.k_out = torch.empty(P, dtype=torch.int64, device=dev)
        self.err = torch.empty(P, dtype=torch.float64, device=dev)
        self.status = torch.empty(P, dtype=torch.int32, device=dev)
        self.xp = (ctypes.c_void_p * P)(*[X.data_ptr() for X in Xs])
        self.sp = (ctypes.c_void_p * P)(*[t.data_ptr() for t in self.S])
        self.wpp = (ctypes.c_void_p * P)(*[t.data_ptr() for t in self.W])
        self.device = dev
        self._lib = L
        self.h = None
        if not handle:
            return
        s = self._stream(stream)
        h = ctypes.c_void_p(0)
        st = L.rbrp_batch_create(P, self.xp, self.m, self.n, self.fp64_in, ctypes.byref(self.opts),
                                 ctypes.c_void_p(self.wp), self.need, self.sp, self.wpp,
                                 ctypes.c_void_p(self.k_out.data_ptr()), ctypes.c_void_p(self.err.data_ptr()),
                                 ctypes.c_void_p(self.status.data_ptr()), ctypes.c_void_p(s.cuda_stream),
                                 ctypes.byref(h))
        _check(st, "rbrp_batch_create", allow_notconverged=False)
        self.h = h

    def _stream(self, stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream(self.device)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self._lib.rbrp_batch_destroy(h)
            self.h = None

    def run(self, tol, stream=None):
        """Queue one batched solve on the stream (no synchronisation)."""
        st = self._lib.rbrp_batch_run(self.h, float(tol), ctypes.c_void_p(self._stream(stream).cuda_stream))
        _check(st, "rbrp_batch_run", allow_notconverged=False)

    def run_once(self, tol, stream=None):
        """One solve through the single-call entry point rbrp_id_batched (no handle)."""
        st = self._lib.rbrp_id_batched(self.P, self.xp, self.m, self.n, self.fp64_in, float(tol),
                                       ctypes.byref(self.opts), ctypes.c_void_p(self.wp), self.need, self.sp,
                                       self.wpp, ctypes.c_void_p(self.k_out.data_ptr()),
                                       ctypes.c_void_p(self.err.data_ptr()), ctypes.c_void_p(self.status.data_ptr()),
                                       ctypes.c_void_p(self._stream(stream).cuda_stream))
        _check(st, "rbrp_id_batched", allow_notconverged=False)

    def graph(self, tol):
        """A torch.cuda.CUDAGraph holding one solve at tol (replay() re-solves every problem)."""
        import torch
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self.run(float(tol), side)
        torch.cuda.current_stream(self.device).wait_stream(side)
        return g

    def tune(self, tol, reps=2, stream=None):
        """Time every schedule that fits, bucket by bucket, keep the fastest; returns bucket 0's
        schedule, the per-bucket schedules (buckets) and the ms per run summed over buckets."""
        best = ctypes.c_float(0.0)
        st = self._lib.rbrp_batch_autotune(self.h, float(tol), int(reps),
                                           ctypes.c_void_p(self._stream(stream).cuda_stream), ctypes.byref(best))
        _check(st, "rbrp_batch_autotune", allow_notconverged=False)
        out = self.schedule()
        out["buckets"] = self.buckets()
        out["ms"] = float(best.value)
        return out

    def buckets(self):
        """Per-shape buckets: problems, largest n and schedule (threads, ctas_per_sm, vec, ctas) of each."""
        out = []
        for i in range(int(self._lib.rbrp_batch_buckets(self.h))):
            pr, t, p, v, c = (ctypes.c_int32(0) for _ in range(5))
            nm = ctypes.c_int64(0)
            _check(self._lib.rbrp_batch_get_bucket(self.h, i, ctypes.byref(pr), ctypes.byref(nm), ctypes.byref(t),
                                                   ctypes.byref(p), ctypes.byref(v), ctypes.byref(c)),
                   "rbrp_batch_get_bucket", allow_notconverged=False)
            out.append(dict(problems=pr.value, n_max=nm.value, threads=t.value, ctas_per_sm=p.value, vec=v.value,
                            ctas=c.value))
        return out

    def set_bucket_schedule(self, i, threads, ctas_per_sm, vec):
        _check(self._lib.rbrp_batch_set_bucket_schedule(self.h, int(i), int(threads), int(ctas_per_sm), int(vec)),
               "rbrp_batch_set_bucket_schedule", allow_notconverged=False)

    def schedule(self):
        t, p, c = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self._lib.rbrp_batch_get_schedule(self.h, ctypes.byref(t), ctypes.byref(p), ctypes.byref(c)),
               "rbrp_batch_get_schedule", allow_notconverged=False)
        return dict(threads=t.value, ctas_per_sm=p.value, ctas=c.value)

    def set_schedule(self, threads, ctas_per_sm):
        _check(self._lib.rbrp_batch_set_schedule(self.h, int(threads), int(ctas_per_sm)), "rbrp_batch_set_schedule",
               allow_notconverged=False)

    def results(self):
        ks, es, ss = self.k_out.tolist(), self.err.tolist(), self.status.tolist()
        out = []
        for p in range(self.P):
            k = int(ks[p])
            out.append(dict(S=self.S[p][:k], W=self.W[p][:, :k], k=k, rel_err_sq=es[p], status=int(ss[p]),
                            converged=(ss[p] == 0)))
        return out


def rbrp_id_batched(Xs, tol, block=16, seed=0, precision="fp32", tau_b=-1.0, k_max=0, sampler="random",
                    stream=None, problem=0):
    """P independent row IDs in one launch (rbrp_id_batched of include/rbrp.h).

    Xs: list of CUDA tensors (all FP32 or all FP64, row-major, m <= 4096 rows,
    n <= 256 columns); problem p uses Philox problem id problem + p.  Returns one dict per
    problem: S (int64 CUDA tensor, acceptance order), W (m x k FP64 CUDA tensor),
    k, rel_err_sq, status.
    """
    import torch
    if len(Xs) == 0:
        return []
    b = Batch(Xs, block, seed, precision, tau_b, k_max, sampler, problem, handle=False)
    s = stream if stream is not None else torch.cuda.current_stream(b.device)
    b.run_once(tol, s)
    s.synchronize()
    return b.results()


# ---------------------------------------------------------------- sketchy pivoting + OSID
def sketch_opts(precision="fp64", block=64, w_precision="fp64", osid_cols=0):
    o = SketchOpts()
    o.precision = PRECISIONS[precision]
    o.block = int(block)
    o.w_precision = W_PRECISIONS[w_precision]
    o.osid_cols = int(osid_cols)
    return o


def rbrp_sketch_workspace_size(n, d, l, k, opts):
    out = ctypes.c_size_t(0)
    st = load().rbrp_sketch_workspace_size(int(n), int(d), int(l), int(k), ctypes.byref(opts), ctypes.byref(out))
    if st != 0:
        raise RBRPError(st, "rbrp_sketch_workspace_size")
    return out.value


class SketchWorkspace:
    """Device buffers for repeated rbrp_sketch_id calls of one shape (allocated once by PyTorch)."""

    def __init__(self, n, d, l, k, opts, device=None):
        import torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.shape = (int(n), int(d), int(l), int(k))
        self.ws = torch.empty(rbrp_sketch_workspace_size(n, d, l, k, opts) + 256, dtype=torch.uint8, device=dev)
        self.skel = torch.empty(int(k), dtype=torch.int64, device=dev)
        self.W = torch.empty((int(n), int(k)), dtype=torch.float64, device=dev)

    def ptr(self):
        return (self.ws.data_ptr() + 255) // 256 * 256

    def nbytes(self):
        return self.ws.numel() - (self.ptr() - self.ws.data_ptr())


def rbrp_sketch_id(X, Omega, k, precision="fp64", block=64, w_precision="fp64", osid_cols=0, workspace=None,
                   stream=None):
    """SkLUPP skeletons and the OSID interpolation matrix (Sec. 3.2, Alg. 4) of a CUDA tensor X
    (n x d) with the caller's embedding Omega (CUDA tensor, d x l: FP64 for precision "fp64",
    else FP32).  Returns dict(S, W (n x |S| FP64), k, blocks, rel_err_sq (sketched), converged)."""
    import torch
    _check_x(X, cuda=True)
    n, d = X.shape
    if Omega.dim() != 2 or not Omega.is_cuda or Omega.device != X.device or not Omega.is_contiguous():
        raise ValueError("Omega must be a contiguous 2-D CUDA tensor on X's device")
    if Omega.shape[0] != d:
        raise ValueError("Omega must have d = %d rows" % d)
    want = torch.float64 if precision == "fp64" else torch.float32
    if Omega.dtype != want:
        raise ValueError("Omega must be %s for precision %s" % (want, precision))
    l = Omega.shape[1]
    opts = sketch_opts(precision, block, w_precision, osid_cols)
    ws = workspace if workspace is not None else SketchWorkspace(n, d, l, k, opts, X.device)
    if ws.shape != (n, d, l, int(k)) or ws.ws.device != X.device:
        raise ValueError("workspace was made for another shape or device")
    res = Result()
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    st = load().rbrp_sketch_id(ctypes.c_void_p(X.data_ptr()), int(X.dtype == torch.float64), n, d, X.stride(0),
                               ctypes.c_void_p(Omega.data_ptr()), l, int(k), ctypes.byref(opts),
                               ctypes.c_void_p(ws.ptr()), ws.nbytes(), ctypes.c_void_p(ws.skel.data_ptr()),
                               ctypes.c_void_p(ws.W.data_ptr()), int(k), ctypes.byref(res),
                               ctypes.c_void_p(s.cuda_stream))
    _check(st, "rbrp_sketch_id")
    out = _result_dict(res, st)
    kk = out["k"]
    out["S"] = ws.skel[:kk]
    out["W"] = ws.W[:, :kk]
    return out


# ---------------------------------------------------------------- row shards of one ID
def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class Shard:
    """Rows [row_base, row_base + n_local) of one ID on this GPU (include/rbrp.h, row shards).

    X_local: CUDA tensor (n_local x d, FP32/FP64); k_cap: the whole ID's min(n, d, k_max).
    The per-block steps are draw(), rows(), block(); after the loop l_rows() and w().  Host
    arrays are numpy (the caller exchanges them between shards); sum_sq = this shard's
    ||X_local||_F^2."""

    def __init__(self, X_local, row_base, k_cap, block=16, precision="fp64", seed=0, problem=0, sampler="random",
                 tau_b=-1.0, chain="default", w_precision="fp64", stream=None):
        import torch
        _check_x(X_local, cuda=True)
        self.X = X_local
        self.n, self.d = X_local.shape
        self.row_base = int(row_base)
        self.k_cap = int(k_cap)
        self.block_size = int(block)
        self.opts = make_opts(block, precision, tau_b, k_cap, seed, problem, sampler, w_precision, "residual", chain)
        out = ctypes.c_size_t(0)
        st = load().rbrp_shard_workspace_size(self.n, self.d, self.k_cap, ctypes.byref(self.opts), ctypes.byref(out))
        if st != 0:
            raise RBRPError(st, "rbrp_shard_workspace_size")
        self.ws = torch.empty(out.value + 256, dtype=torch.uint8, device=X_local.device)
        ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(X_local.device)
        self.h = ctypes.c_void_p()
        ss = ctypes.c_double(0.0)
        st = load().rbrp_shard_create(ctypes.c_void_p(X_local.data_ptr()), int(X_local.dtype == torch.float64),
                                      self.n, self.d, X_local.stride(0), self.row_base, self.k_cap,
                                      ctypes.byref(self.opts), ctypes.c_void_p(ptr),
                                      self.ws.numel() - (ptr - self.ws.data_ptr()),
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h), ctypes.byref(ss))
        _check(st, "rbrp_shard_create", allow_notconverged=False)
        self.sum_sq = ss.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None and self.h.value:
            _lib.rbrp_shard_destroy(self.h)
            self.h = ctypes.c_void_p()

    def draw(self):
        rows = np.zeros(256, dtype=np.int64)
        keys = np.zeros(256, dtype=np.float64)
        cnt = ctypes.c_int64(0)
        _check(load().rbrp_shard_draw(self.h, _p64(rows), _pd(keys), ctypes.byref(cnt)), "rbrp_shard_draw", False)
        return rows[:cnt.value].copy(), keys[:cnt.value].copy()

    def rows(self, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        V = np.zeros((len(rows), self.d), dtype=np.float64)
        own = np.zeros(len(rows), dtype=np.int32)
        _check(load().rbrp_shard_rows(self.h, _p64(rows), len(rows), _pd(V), _p32(own)), "rbrp_shard_rows", False)
        return V, own.astype(bool)

    def block(self, V, S_t):
        V = np.ascontiguousarray(V, dtype=np.float64)
        S_t = np.ascontiguousarray(S_t, dtype=np.int64)
        acc = np.zeros(len(S_t), dtype=np.int64)
        bp = ctypes.c_int64(0)
        dsum = ctypes.c_double(0.0)
        st = load().rbrp_shard_block(self.h, _pd(V), _p64(S_t), len(S_t), _p64(acc), ctypes.byref(bp),
                                     ctypes.byref(dsum))
        _check(st, "rbrp_shard_block", False)
        return acc[:bp.value].copy(), dsum.value

    def l_rows(self, rows, k):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        Lr = np.zeros((len(rows), int(k)), dtype=np.float64)
        own = np.zeros(len(rows), dtype=np.int32)
        st = load().rbrp_shard_l_rows(self.h, _p64(rows), len(rows), int(k), _pd(Lr), _p32(own))
        _check(st, "rbrp_shard_l_rows", False)
        return Lr, own.astype(bool)

    def w(self, L1, skel):
        import torch
        L1 = np.ascontiguousarray(L1, dtype=np.float64)
        skel = np.ascontiguousarray(skel, dtype=np.int64)
        k = len(skel)
        W = torch.empty((self.n, max(k, 1)), dtype=torch.float64, device=self.X.device)
        st = load().rbrp_shard_w(self.h, _pd(L1), _p64(skel), k, ctypes.c_void_p(W.data_ptr()), max(k, 1))
        _check(st, "rbrp_shard_w", False)
        return W[:, :k]
