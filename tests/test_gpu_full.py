"""GPU parity at the full sizes of the configurations (R-MAT scale 20 and
22, the 4096 x 4096 grid), through the same C-ABI path the benchmark times.
Every batch of every trajectory is compared with the oracle (parent arrays
bit for bit, labels, the exact checker, the counters); the oracle checks run
side by side in a process pool (tests/oracle_pool.py)."""
import pytest
import torch

import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import run_trajectory_pooled

pytestmark = pytest.mark.gpu

I, D = drsf.INSERT, drsf.DELETE


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()


def test_rmat20_batch_sizes():
    """R-MAT scale 20, edge factor 16, seed 2: for each batch size 10K, 100K
    and 1M in turn, 20 batches alternating insert and delete (deletes half
    tree edges) on the evolving graph."""
    g = workloads.rmat_graph(20, 16, seed=2)
    sched = [(I if k % 2 == 0 else D, b) for b in (10_000, 100_000, 1_000_000) for k in range(20)]
    assert run_trajectory_pooled(g, sched, seed=2) == 60


def test_grid4096_deep():
    """4096 x 4096 grid, p = 0.6, 0.1% shortcuts, seed 3: 100K deletes with 90%
    tree edges (deep re-rooted paths), then 100K local inserts, twice."""
    g = workloads.grid_graph(4096, 4096, seed=3)
    assert run_trajectory_pooled(g, [(D, 100_000), (I, 100_000)] * 2, seed=3, tree_frac=0.9, local=64) == 4


def test_grid4096_euler_reversal():
    """The same deep-grid batches with the Euler-tour path reversal
    (Algorithm 3) in place of walks and doubling marks."""
    g = workloads.grid_graph(4096, 4096, seed=3)
    assert run_trajectory_pooled(g, [(D, 100_000), (I, 100_000)], seed=3, tree_frac=0.9, local=64,
                                 flags=drsf.DETERMINISTIC | drsf.EULER_REVERSAL) == 2


@pytest.fixture(scope="module")
def rmat22():
    return workloads.rmat_graph(22, 16, seed=5)


def test_rmat22_bench_trajectory(rmat22):
    """R-MAT scale 22 (the benchmark workload), the benchmark's own
    trajectory (seed 5): its first 8 steps of one 100K insert batch and one
    100K delete batch."""
    g = rmat22
    assert run_trajectory_pooled(g, [(I, 100_000), (D, 100_000)] * 8, seed=5) == 16


@pytest.mark.parametrize("variant", ["sg", "hs"])
def test_rmat22_replacement_variants(variant, rmat22):
    """The benchmark trajectory's first two steps with each replacement-edge
    variant forced (the default picks HS for these inserts and SG for these
    deletes): same forests as the oracle."""
    g = rmat22
    flags = drsf.DETERMINISTIC | (drsf.REPL_SG if variant == "sg" else drsf.REPL_HS)
    assert run_trajectory_pooled(g, [(I, 100_000), (D, 100_000)] * 2, seed=5, flags=flags) == 4
