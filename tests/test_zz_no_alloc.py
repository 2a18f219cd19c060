"""The allocation-free labelling entry point, through the C ABI.

drsf_forest_labels_noalloc serves callers that cannot allocate device memory
when they need the answer; its scratch is a fixed array inside the library.
Its labels must equal those of the existing entry point drsf_labels on the
same forest, exactly (integer output), on two calls in a row (the second call
must not see the first call's leftovers).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import dev_tensor, make_forest

pytestmark = pytest.mark.gpu


def _noalloc(lib, parent_dev, out_dev):
    fn = lib.drsf_forest_labels_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn(parent_dev.numel(), parent_dev.data_ptr(), out_dev.data_ptr(),
              torch.cuda.current_stream().cuda_stream)


def test_noalloc_labels_match_drsf_labels_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    lib = drsf.library()
    cases = [workloads.rmat_graph(17, 8, seed=31), workloads.er_graph(20_000, 25_000, seed=32)]
    for g in cases:   # two calls in a row, different sizes and forests
        f = make_forest(g)
        tr = workloads.Trajectory(g, seed=33)
        f.delete(dev_tensor(tr.next_batch(drsf.DELETE, 2000)))
        parent = f.parent()
        want = f.labels().cpu().numpy()
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(lib, parent, out) == drsf.OK
        assert np.array_equal(out.cpu().numpy(), want)
        f.close()


def test_noalloc_rejects_oversize_and_bad_parent():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = drsf.library()
    big = torch.zeros(lib_max() + 1, dtype=torch.int32, device="cuda")
    out = torch.empty_like(big)
    assert _noalloc(lib, big, out) == drsf.EINVAL
    bad = dev_tensor(np.array([0, 5, 1], np.int32))
    assert _noalloc(lib, bad, torch.empty(3, dtype=torch.int32, device="cuda")) == drsf.EINVAL
    ok = dev_tensor(np.array([0, 0, 1, 3], np.int32))
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, ok, out) == drsf.OK
    assert out.cpu().tolist() == [0, 0, 0, 3]


def lib_max():
    return 1 << 20
