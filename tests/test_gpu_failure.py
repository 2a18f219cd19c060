"""Failure detection on the GPU without a fault: a grid barrier whose peer
never arrives gives up after its bounded wait, reports DRSF_ETIMEOUT, and the
CUDA context stays usable (a normal update still matches the oracle)."""
import numpy as np
import pytest
import torch

import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import check_batch, make_forest

pytestmark = pytest.mark.gpu


def test_barrier_wait_times_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    assert drsf.selftest_barrier_timeout() == drsf.ETIMEOUT
    g = workloads.er_graph(3000, 4000, seed=21)
    f = make_forest(g)
    tr = workloads.Trajectory(g, seed=22)
    check_batch(f, g.n, g.keys, g.parent, drsf.DELETE, tr.next_batch(drsf.DELETE, 500))
    f.close()
