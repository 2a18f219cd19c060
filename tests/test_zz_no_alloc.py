"""The allocation-free labelling entry point, through the C ABI.

drsf_forest_labels_noalloc serves callers that cannot allocate device memory
when they need the answer (a device budget fixed up front, code running
inside an allocator's callbacks, loops where cudaMalloc would synchronise);
its scratch is a fixed array inside the library.  Its labels must equal those
of the existing entry point drsf_labels on the same forest, and the oracle's
component minima of the forest's own edge set, exactly (integer output), on
several calls in a row: a smaller graph after a larger one, then the larger
graph again with a different forest, so leftovers of an earlier call in the
shared array would show.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import dev_tensor, make_forest

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20   # DRSF_NOALLOC_MAX_N


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()


def _noalloc(parent_dev, out_dev):
    fn = drsf.library().drsf_forest_labels_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn(parent_dev.numel(), parent_dev.data_ptr(), out_dev.data_ptr(),
              torch.cuda.current_stream().cuda_stream)


def _forest_keys(parent):
    """Edge keys (min << 32 | max) of the tree edges of a parent array."""
    v = np.arange(len(parent), dtype=np.int64)
    p = parent.astype(np.int64)
    sel = p != v
    lo, hi = np.minimum(v[sel], p[sel]), np.maximum(v[sel], p[sel])
    return np.unique((lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64))


def test_noalloc_labels_match_drsf_labels_and_oracle():
    big = workloads.rmat_graph(17, 8, seed=31)
    small = workloads.er_graph(20_000, 25_000, seed=32)
    # large graph, smaller graph, then the large graph again after another
    # delete batch (a different forest on the same n)
    for g, n_del in ((big, 2000), (small, 2000), (big, 6000)):
        f = make_forest(g)
        tr = workloads.Trajectory(g, seed=33 + n_del)
        f.delete(dev_tensor(tr.next_batch(drsf.DELETE, n_del)))
        parent = f.parent()
        want = f.labels().cpu().numpy()
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(parent, out) == drsf.OK
        got = out.cpu().numpy()
        assert np.array_equal(got, want)
        par = parent.cpu().numpy()
        assert np.array_equal(got, oracle.labels(g.n, _forest_keys(par)))
        f.close()


def test_noalloc_rejects_oversize():
    big = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    assert _noalloc(big, torch.empty_like(big)) == drsf.EINVAL


def test_noalloc_bad_parent_ids_and_cycles():
    out3 = torch.empty(3, dtype=torch.int32, device="cuda")
    assert _noalloc(dev_tensor(np.array([0, 5, 1], np.int32)), out3) == drsf.EINVAL
    assert _noalloc(dev_tensor(np.array([0, -1, 1], np.int32)), out3) == drsf.EINVAL
    # a 2-cycle and a 3-cycle (no root reachable)
    out2 = torch.empty(2, dtype=torch.int32, device="cuda")
    assert _noalloc(dev_tensor(np.array([1, 0], np.int32)), out2) == drsf.EINVAL
    assert _noalloc(dev_tensor(np.array([1, 2, 0], np.int32)), out3) == drsf.EINVAL
    # a tree hanging off a 3-cycle
    assert _noalloc(dev_tensor(np.array([1, 2, 0, 0, 3], np.int32)),
                    torch.empty(5, dtype=torch.int32, device="cuda")) == drsf.EINVAL
    # many blocks: a bad id or a cycle in the last block of a 2^20 array must
    # be reported, whichever block runs first
    par = np.arange(MAX_N, dtype=np.int32) // 2   # a binary tree rooted at 0
    out = torch.empty(MAX_N, dtype=torch.int32, device="cuda")
    bad = par.copy()
    bad[MAX_N - 1] = MAX_N
    assert _noalloc(dev_tensor(bad), out) == drsf.EINVAL
    cyc = par.copy()
    cyc[MAX_N - 3:] = [MAX_N - 2, MAX_N - 1, MAX_N - 3]
    assert _noalloc(dev_tensor(cyc), out) == drsf.EINVAL
    # the status word does not stick: a valid forest right after is accepted
    assert _noalloc(dev_tensor(par), out) == drsf.OK
    assert np.array_equal(out.cpu().numpy(), np.zeros(MAX_N, np.int32))
    ok = dev_tensor(np.array([0, 0, 1, 3], np.int32))
    out4 = torch.empty(4, dtype=torch.int32, device="cuda")
    assert _noalloc(ok, out4) == drsf.OK
    assert out4.cpu().tolist() == [0, 0, 0, 3]
