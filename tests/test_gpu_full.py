"""GPU parity at the full sizes of the configurations (R-MAT scale 20 and
22, the 4096 x 4096 grid), through the same C-ABI path the benchmark times.
The oracle handles these sizes in seconds per batch, so every output is
compared, not a sample."""
import pytest
import torch

import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import run_trajectory

pytestmark = pytest.mark.gpu

I, D = drsf.INSERT, drsf.DELETE


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()


def test_rmat20_batch_sizes():
    """R-MAT scale 20, edge factor 16, seed 2: insert/delete at 10K, 100K, 1M."""
    g = workloads.rmat_graph(20, 16, seed=2)
    run_trajectory(g, [(I, 10_000), (D, 10_000), (I, 100_000), (D, 100_000), (I, 1_000_000),
                       (D, 1_000_000)], seed=2, labels=False)


def test_grid4096_deep():
    """4096 x 4096 grid, p = 0.6, 0.1% shortcuts, seed 3: 100K deletes with 90%
    tree edges, then 100K local inserts."""
    g = workloads.grid_graph(4096, 4096, seed=3)
    run_trajectory(g, [(D, 100_000), (I, 100_000)], seed=3, tree_frac=0.9, local=64, labels=False)


def test_rmat22_100k():
    """R-MAT scale 22 (the benchmark workload), 100K insert then 100K delete."""
    g = workloads.rmat_graph(22, 16, seed=5)
    run_trajectory(g, [(I, 100_000), (D, 100_000)], seed=5, labels=False)
