"""The static from-scratch rebuild (components + multi-source BFS from the
component minima), the plain alternative to the dynamic update: its forest
must pass the exact checker for the current graph and its labels must equal
the oracle's component minima; the handle's own forest is left untouched."""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import check_batch, make_forest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()


def _check_static(f, n, keys):
    before = f.parent().cpu().numpy()
    par, lab, levels = f.static_forest(with_levels=True)
    par = par.cpu().numpy()
    lab = lab.cpu().numpy()
    assert oracle.check_forest(n, keys, par) == 0
    want = oracle.labels(n, keys)
    assert np.array_equal(lab, want)
    roots = np.nonzero(par == np.arange(n))[0]
    assert np.array_equal(np.sort(roots), np.unique(want))
    assert np.array_equal(f.parent().cpu().numpy(), before)
    assert levels >= 1


@pytest.mark.parametrize("make", [
    lambda: workloads.er_graph(20_000, 25_000, seed=1),
    lambda: workloads.rmat_graph(16, 16, seed=2),
    lambda: workloads.grid_graph(256, 256, seed=3),
])
def test_static_forest_valid(make):
    g = make()
    f = make_forest(g)
    _check_static(f, g.n, g.keys)
    # after updates (incl. overflow edges from a large insert)
    keys, par = g.keys, g.parent
    tr = workloads.Trajectory(g, seed=9)
    for op, b in [(drsf.INSERT, max(g.m // 4, 100)), (drsf.DELETE, max(g.m // 10, 100))]:
        batch = tr.next_batch(op, b)
        keys, par, _ = check_batch(f, g.n, keys, par, op, batch, labels=False)
        tr.advance(batch, op, par)
    _check_static(f, g.n, keys)
    f.close()


def test_static_forest_rmat22():
    g = workloads.rmat_graph(22, 16, seed=5)
    f = make_forest(g)
    _check_static(f, g.n, g.keys)
    f.close()
