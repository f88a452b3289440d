"""CPU checks of the Python binding's buffer validation: every buffer handed to the C ABI is
checked (dtype, device, shape, layout) before the call, because the library receives plain
pointers and would otherwise read or write past a wrong one.  Each case raises before any
CUDA call or device allocation."""
import numpy as np
import pytest
import torch

from paper_2309_16002_gb300 import rbrp as R


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()
    R.load()


def test_device_entry_points_want_cuda_float_inputs():
    X = torch.zeros((50, 10), dtype=torch.float32)  # host tensor
    with pytest.raises(ValueError):
        R.rbrp_id(X, 1e-3)
    with pytest.raises(ValueError):
        R.rbrp_id_noalloc(X, 1e-3, torch.empty(10, dtype=torch.int64), torch.empty((50, 10), dtype=torch.float64))


@pytest.mark.parametrize("dtype", [np.float16, np.int32, np.complex64])
def test_host_entry_point_rejects_other_dtypes(dtype):
    X = np.zeros((50, 10), dtype=dtype)
    with pytest.raises(ValueError):
        R.rbrp_id_host(X, 1e-3)


def test_host_entry_point_checks_its_outputs():
    X = np.zeros((50, 10), dtype=np.float32)
    good_s = torch.empty(10, dtype=torch.int64)
    good_W = torch.empty((50, 10), dtype=torch.float64)
    bad = [
        (torch.empty(9, dtype=torch.int64), good_W),                 # skel shorter than k_cap
        (torch.empty(10, dtype=torch.int32), good_W),                # skel not int64
        (good_s, torch.empty((49, 10), dtype=torch.float64)),        # W missing a row
        (good_s, torch.empty((50, 11), dtype=torch.float64)),        # W pitch is not k_cap
        (good_s, torch.empty((50, 10), dtype=torch.float32)),        # W not float64
        (good_s, torch.empty((10, 50), dtype=torch.float64).t()),    # W not C-contiguous
    ]
    for s, W in bad:
        with pytest.raises(ValueError):
            R.rbrp_id_host(X, 1e-3, skel_out=s, W_out=W)
    # with k_max the outputs are sized for k_cap = k_max
    with pytest.raises(ValueError):
        R.rbrp_id_host(X, 1e-3, k_max=4, skel_out=good_s, W_out=good_W)


def test_host_entry_point_wants_a_contiguous_2d_array():
    with pytest.raises(ValueError):
        R.rbrp_id_host(np.zeros((10, 50), dtype=np.float32).T, 1e-3)
    with pytest.raises(ValueError):
        R.rbrp_id_host(np.zeros(50, dtype=np.float32), 1e-3)
    with pytest.raises(ValueError):
        R.rbrp_id_host(np.zeros((0, 5), dtype=np.float32), 1e-3)


def test_batch_wants_one_float_dtype_on_cuda():
    with pytest.raises(ValueError):
        R.Batch([])
    with pytest.raises(ValueError):
        R.Batch([torch.zeros((20, 5), dtype=torch.float16)])
    with pytest.raises(ValueError):
        R.Batch([torch.zeros((20, 5), dtype=torch.float32)])        # host tensor
