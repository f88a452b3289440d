"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every
function declared in include/rbrp.h (no compute calls: there may be no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rbrp_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g
    g.build()
    from paper_2309_16002_gb300 import rbrp
    return rbrp.lib_path()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("rbrp_id", "rbrp_workspace_size", "rbrp_id_host", "rbrp_default_opts"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    from paper_2309_16002_gb300 import rbrp
    L = rbrp.load()
    for name in declared_functions():
        assert hasattr(L, name)
    assert set(rbrp.exported_symbols()) <= declared_functions()


def test_workspace_size_and_validation_on_host(libpath):
    """Pure host logic of the ABI (no GPU needed): sizing and argument validation."""
    from paper_2309_16002_gb300 import rbrp
    o = rbrp.make_opts(block=64, precision="tf32")
    ws = rbrp.rbrp_workspace_size(100000, 1000, o)
    # at least R (FP32) + L (FP32, n x k_cap) + Q (FP64, k_cap x d)
    assert ws >= 100000 * 1024 * 4 + 100000 * 1000 * 4 + 1000 * 1024 * 8
    with pytest.raises(rbrp.RBRPError):
        rbrp.rbrp_workspace_size(100, 10, rbrp.make_opts(block=0))
    with pytest.raises(rbrp.RBRPError):
        rbrp.rbrp_workspace_size(100, 10, rbrp.make_opts(block=300, precision="fp64"))
    with pytest.raises(rbrp.RBRPError):   # the FP32 filter of the plain TF32 chain: b <= 128
        rbrp.rbrp_workspace_size(100, 10, rbrp.make_opts(block=256, precision="tf32"))
    # wider blocks run as column chunks of Q': 3xTF32 and the FP64 chain take b <= 256
    assert rbrp.rbrp_workspace_size(100, 10, rbrp.make_opts(block=256, precision="tf32x3")) > 0
    assert rbrp.rbrp_workspace_size(100, 10, rbrp.make_opts(block=256, precision="tf32", chain="fp64")) > 0
    # the downdate form: FP64 only, and it keeps no residual copy of X
    with pytest.raises(rbrp.RBRPError):
        rbrp.rbrp_workspace_size(100, 10, rbrp.make_opts(precision="tf32", form="downdate"))
    res = rbrp.rbrp_workspace_size(100000, 1000, rbrp.make_opts(precision="fp64"))
    dd = rbrp.rbrp_workspace_size(100000, 1000, rbrp.make_opts(precision="fp64", form="downdate"))
    assert res - dd >= 100000 * 1000 * 8
    with pytest.raises(rbrp.RBRPError):
        rbrp.rbrp_workspace_size(0, 10, o)
    # the FP64 chain beside the TF32 update: accepted, and it needs no less than the FP32 chain
    # but for the FP32 chain's Gram partials (ceil(d / 64) tiles of 64 x 64 FP32)
    c64 = rbrp.rbrp_workspace_size(100000, 1000, rbrp.make_opts(block=64, precision="tf32", chain="fp64"))
    assert c64 >= ws - 16 * 64 * 64 * 4
    bad = rbrp.make_opts(block=64, precision="tf32")
    bad.chain = 2
    with pytest.raises(rbrp.RBRPError):
        rbrp.rbrp_workspace_size(100, 10, bad)
    assert rbrp.rbrp_host_workspace_size(1000, 50, 0, o) > rbrp.rbrp_workspace_size(1000, 50, o)


def test_status_strings(libpath):
    from paper_2309_16002_gb300 import rbrp
    L = rbrp.load()
    assert L.rbrp_status_string(0) == b"ok"
    assert b"workspace" in L.rbrp_status_string(7)


def test_batched_workspace_validation_on_host(libpath):
    """Host logic of the batched entry points: sizes and limits, no GPU needed."""
    import ctypes
    from paper_2309_16002_gb300 import rbrp
    L = rbrp.load()

    def size(ms, ns, **kw):
        P = len(ms)
        m = (ctypes.c_int64 * max(P, 1))(*ms)
        n = (ctypes.c_int64 * max(P, 1))(*ns)
        o = rbrp.make_opts(**kw)
        out = ctypes.c_size_t(0)
        st = L.rbrp_batched_workspace_size(P, m, n, ctypes.byref(o), ctypes.byref(out))
        return st, out.value

    st, a = size([100, 2000], [30, 256], block=16, precision="fp32")
    assert st == 0 and a > 0
    # one slot per resident CTA of the largest schedule, each for the largest problem
    st, b = size([100, 2000, 50], [30, 256, 10], block=16, precision="fp32")
    assert st == 0 and b >= a
    st64, c = size([100, 2000], [30, 256], block=16, precision="fp64")
    assert st64 == 0 and c > a
    assert size([4097], [10], block=16, precision="fp32")[0] == 1   # m > 4096
    assert size([10], [257], block=16, precision="fp32")[0] == 1    # n > 256
    assert size([10], [10], block=33, precision="fp32")[0] == 1     # b > 32
    assert size([0], [10], block=16, precision="fp32")[0] == 1      # empty problem
    assert size([10], [10], block=8, precision="fp32", sampler="greedy_exact")[0] == 0
    assert size([], [], block=8, precision="fp32")[0] == 0          # P = 0 is valid (nothing to do)


def test_opts_layout_matches_the_header(libpath):
    """rbrp_default_opts fills every field the binding declares (same layout as rbrp.h)."""
    import ctypes
    from paper_2309_16002_gb300 import rbrp
    o = rbrp.Opts()
    ctypes.memset(ctypes.byref(o), 0xAB, ctypes.sizeof(o))
    rbrp.load().rbrp_default_opts(ctypes.byref(o))
    assert (o.precision, o.block, o.tau_b, o.k_max, o.seed, o.problem) == (1, 64, -1.0, 0, 0, 0)
    assert (o.sampler, o.w_precision, o.form, o.chain) == (0, 0, 0, 0)


def test_sketch_workspace_validation_on_host(libpath):
    """Host logic of rbrp_sketch_workspace_size: sizes, limits and options, no GPU needed."""
    from paper_2309_16002_gb300 import rbrp
    o = rbrp.sketch_opts(precision="tf32", block=64)
    a = rbrp.rbrp_sketch_workspace_size(100000, 1000, 300, 100, o)
    # at least the sketch Y (FP32, n x l) and the LUPP copy of its first k columns
    assert a >= 100000 * 300 * 4 + 100000 * 100 * 4
    b = rbrp.rbrp_sketch_workspace_size(100000, 1000, 300, 100, rbrp.sketch_opts(precision="fp64", block=64))
    assert b > a
    for bad in [(100, 10, 5, 6), (100, 10, 0, 1), (5, 10, 8, 6), (0, 10, 5, 2)]:  # k > l, l < 1, k > n, n < 1
        with pytest.raises(rbrp.RBRPError):
            rbrp.rbrp_sketch_workspace_size(*bad, o)
    with pytest.raises(rbrp.RBRPError):   # osid_cols outside [k, l]
        rbrp.rbrp_sketch_workspace_size(1000, 50, 30, 10, rbrp.sketch_opts(osid_cols=5))
    with pytest.raises(rbrp.RBRPError):   # b <= 256
        rbrp.rbrp_sketch_workspace_size(1000, 50, 30, 10, rbrp.sketch_opts(precision="tf32", block=300))
    assert rbrp.rbrp_sketch_workspace_size(1000, 50, 30, 10, rbrp.sketch_opts(osid_cols=10)) > 0
