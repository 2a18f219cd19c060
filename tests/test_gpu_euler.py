"""Path reversal by Euler-tour intervals (Algorithm 3, DRSF_EULER_REVERSAL)
must give exactly the oracle's forest, like the pointer-doubling marks."""
import numpy as np
import pytest
import torch

import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import check_batch, dev_tensor, make_forest, run_trajectory, _tiny_graph

pytestmark = pytest.mark.gpu

I, D = drsf.INSERT, drsf.DELETE
ET = drsf.DETERMINISTIC | drsf.EULER_REVERSAL


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()


def test_euler_er():
    g = workloads.er_graph(20_000, 25_000, seed=1)
    run_trajectory(g, [(I, 2000), (D, 2000)] * 3, seed=1, flags=ET)


def test_euler_rmat():
    g = workloads.rmat_graph(16, 16, seed=2)
    run_trajectory(g, [(I, 10_000), (D, 10_000)] * 3, seed=3, flags=ET)


def test_euler_grid_deep():
    g = workloads.grid_graph(512, 512, seed=3)
    run_trajectory(g, [(D, 5000), (I, 5000)] * 3, seed=4, tree_frac=0.9, local=64, flags=ET)


def test_euler_long_path():
    n = 100_000
    edges = [(i, i + 1) for i in range(n - 1)] + [(0, n - 1)]
    g = _tiny_graph(n, edges, [0] + list(range(n - 1)))
    f = make_forest(g, flags=ET)
    keys, par, st = check_batch(f, n, g.keys, g.parent, D, np.array([[1, 0]], np.int32))
    assert st["reversed"] == n - 2
    f.close()
