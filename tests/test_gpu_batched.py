"""Batched form: many independent graphs updated by one launch sequence over
their disjoint union (vertex ids offset per graph).  The union's result,
split back per graph, must equal each graph's own oracle result bit for bit,
and each graph's own GPU handle's result."""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import dev_tensor, make_forest

pytestmark = pytest.mark.gpu


def test_union_equals_per_graph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    graphs = workloads.batched_graphs(24, seed=44, n_lo=500, n_hi=30_000)
    budgets = workloads.batched_budgets(graphs, seed=44)
    U = workloads.Union(graphs)
    fu = drsf.DynamicForest(U.n, dev_tensor(workloads.keys_to_edges(U.keys)), dev_tensor(U.parent))
    trs = [workloads.Trajectory(g, seed=1000 + i) for i, g in enumerate(graphs)]
    # insert: one union batch
    ins = [tr.next_batch(drsf.INSERT, b[0]) for tr, b in zip(trs, budgets)]
    fu.insert(dev_tensor(np.concatenate([U.shift(i, b) for i, b in enumerate(ins)])))
    refs = [oracle.apply(g.n, g.keys, g.parent, 0, b, want_keys=True) for g, b in zip(graphs, ins)]
    got = U.split(fu.parent().cpu().numpy())
    for i, r in enumerate(refs):
        assert np.array_equal(got[i], r.parent), i
        trs[i].advance(ins[i], 0, r.parent)
    # delete: one union batch drawn from each graph's state after the insert
    dels = [tr.next_batch(drsf.DELETE, b[1]) for tr, b in zip(trs, budgets)]
    fu.delete(dev_tensor(np.concatenate([U.shift(i, b) for i, b in enumerate(dels)])))
    got = U.split(fu.parent().cpu().numpy())
    lab = U.split(fu.labels().cpu().numpy())
    for i, (g, r0, d) in enumerate(zip(graphs, refs, dels)):
        r = oracle.apply(g.n, r0.keys, r0.parent, 1, d, want_keys=True)
        assert np.array_equal(got[i], r.parent), i
        assert np.array_equal(lab[i], oracle.labels(g.n, r.keys)), i
        # and the graph's own handle gives the same forest
        f = make_forest(g)
        f.insert(dev_tensor(ins[i]))
        f.delete(dev_tensor(d))
        assert np.array_equal(f.parent().cpu().numpy(), r.parent), i
        f.close()
    fu.close()


def test_union_256_graphs_config_shape():
    """The batched configuration at its real shape: 256 graphs (n
    log-uniform in [1K, 256K], half Erdos-Renyi, half R-MAT, seed 4), two
    steps of one insert batch and one delete batch per graph (1-10% of m,
    60/40), applied as union batches; every graph's forest and labels after
    every batch are checked against its own oracle run (process pool)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests.oracle_pool import TrajectoryCheck
    drsf.build()
    graphs = workloads.batched_graphs(256, seed=4)
    U = workloads.Union(graphs)
    fu = drsf.DynamicForest(U.n, dev_tensor(workloads.keys_to_edges(U.keys)), dev_tensor(U.parent))
    trs = [workloads.Trajectory(g, seed=(4 << 20) + i) for i, g in enumerate(graphs)]
    chks = [TrajectoryCheck(g.n, g.keys, g.parent) for g in graphs]
    try:
        for step in range(2):
            budgets = workloads.batched_budgets(graphs, seed=4 + 7919 * step)
            for op in (drsf.INSERT, drsf.DELETE):
                per = [tr.next_batch(op, b[op]) for tr, b in zip(trs, budgets)]
                fu.apply(op, dev_tensor(np.concatenate([U.shift(i, b) for i, b in enumerate(per)])))
                st = fu.stats()
                assert st["applied"] == sum(len(b) for b in per)
                parts = U.split(fu.parent().cpu().numpy())
                labs = U.split(fu.labels().cpu().numpy())
                for i, (tr, b, p, lab) in enumerate(zip(trs, per, parts, labs)):
                    # per-graph counters are not separable from the union's;
                    # check the per-graph forest, labels and checker only
                    chks[i].add(op, b, p, None, lab)
                    tr.advance(b, op, p)
        for c in chks:
            c.result()
    finally:
        fu.close()
