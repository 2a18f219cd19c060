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


# ---------------------------------------------------------------- persistent per-graph kernels

FULL = 2 ** 31 - 1
CLASS_SETS = [
    drsf.DEFAULT_CLASSES,
    ((FULL, 128, 0, 1),),
    ((4096, 1024, 1, 1), (FULL, 256, 2, 4)),
    ((2000, 512, 0, 2), (10_000, 128, 3, 1), (20_000, 1024, 0, 16), (FULL, 256, 1, 8)),
]


def _offsets(U, per):
    bo = np.zeros(len(per) + 1, np.int64)
    bo[1:] = np.cumsum([len(b) for b in per])
    return U.offsets.astype(np.int64), bo


def _run_persistent(graphs, steps, seed, classes, oracle_check=True, union_check=True):
    """Apply `steps` insert+delete steps to every graph with the persistent
    kernels; compare with each graph's oracle result and with the union path
    on the same union batches, after every batch."""
    from tests.oracle_pool import TrajectoryCheck
    U = workloads.Union(graphs)
    edges_u, par_u = dev_tensor(workloads.keys_to_edges(U.keys)), dev_tensor(U.parent)
    fp = drsf.DynamicForest(U.n, edges_u, par_u)
    fu = drsf.DynamicForest(U.n, edges_u, par_u) if union_check else None
    trs = [workloads.Trajectory(g, seed=seed + i) for i, g in enumerate(graphs)]
    chks = [TrajectoryCheck(g.n, g.keys, g.parent) for g in graphs] if oracle_check else None
    try:
        for step in range(steps):
            budgets = workloads.batched_budgets(graphs, seed=seed + 7919 * step)
            for op in (drsf.INSERT, drsf.DELETE):
                per = [tr.next_batch(op, b[op]) for tr, b in zip(trs, budgets)]
                ub = dev_tensor(np.concatenate([U.shift(i, b) for i, b in enumerate(per)]).reshape(-1, 2))
                vo, bo = _offsets(U, per)
                fp.apply_batched(op, ub, vo, bo, classes)
                st = fp.stats()
                assert st["applied"] <= sum(len(b) for b in per)
                got = fp.parent().cpu().numpy()
                if fu is not None:
                    fu.apply(op, ub)
                    su = fu.stats()
                    assert np.array_equal(got, fu.parent().cpu().numpy())
                    for k in ("applied", "self_loops", "dropped", "tree_cut", "replacement", "edges"):
                        assert st[k] == su[k], (k, st[k], su[k])
                parts = U.split(got)
                labs = U.split(fp.labels().cpu().numpy())
                for i, (tr, b, p, lab) in enumerate(zip(trs, per, parts, labs)):
                    if chks is not None:
                        chks[i].add(op, b, p, None, lab)
                    tr.advance(b, op, p)
        if chks is not None:
            for c in chks:
                c.result()
    finally:
        fp.close()
        if fu is not None:
            fu.close()


@pytest.mark.parametrize("ci", range(len(CLASS_SETS)))
def test_persistent_matches_oracle_and_union(ci):
    """Persistent per-graph kernels (drsf_apply_batched) on 24 graphs (n in
    [500, 30K], half ER, half R-MAT), three steps, several size-class and
    block-size schedules: every graph's forest and labels equal its oracle
    run, and the whole union equals the grid-wide path's result."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    graphs = workloads.batched_graphs(24, seed=44, n_lo=500, n_hi=30_000)
    _run_persistent(graphs, 3, seed=1000 + ci, classes=CLASS_SETS[ci])


def test_persistent_256_graphs_config_shape():
    """The batched configuration at its real shape (256 graphs, seed 4) with
    the persistent kernels: two steps, every graph against its oracle run."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    graphs = workloads.batched_graphs(256, seed=4)
    _run_persistent(graphs, 2, seed=4 << 20, classes=drsf.DEFAULT_CLASSES, union_check=False)


def test_persistent_overflow_and_edge_cases():
    """Rows that overflow (many inserts at a star's centre), then deletes
    that cut the star (the overflow edges become candidates); a one-vertex
    graph, an edgeless graph and graphs with empty batch slices."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests.gpu_util import _tiny_graph
    drsf.build()
    # a star on 0..199 and a path on 200..299 (its own tree)
    star = _tiny_graph(300, [(0, i) for i in range(1, 200)] + [(i, i + 1) for i in range(200, 299)], None)
    path = _tiny_graph(200, [(i, i + 1) for i in range(199)], None)
    one = _tiny_graph(1, [], None)
    empty = _tiny_graph(50, [], None)
    er = workloads.er_graph(3000, 4000, seed=9)
    graphs = [star, one, path, empty, er]
    U = workloads.Union(graphs)
    fp = drsf.DynamicForest(U.n, dev_tensor(workloads.keys_to_edges(U.keys)), dev_tensor(U.parent))
    keys = [g.keys for g in graphs]
    pars = [g.parent for g in graphs]
    rng = np.random.default_rng(3)
    ins = [np.array([(0, v) for v in range(200, 300)], np.int32),           # overflow at the centre
           np.zeros((0, 2), np.int32),
           np.array([(0, 199), (5, 150), (3, 3)], np.int32),                # a cycle, a self-loop
           np.array([(i, i + 1) for i in range(0, 49, 2)], np.int32),
           rng.integers(0, 3000, (300, 2)).astype(np.int32)]
    # cut the path into pieces whose cross edges to the centre partly sit in
    # the overflow list; also delete star edges and some of the new edges
    dels = [np.array([(0, v) for v in range(1, 200, 3)] + [(i, i + 1) for i in range(200, 299, 5)] +
                     [(0, v) for v in range(203, 300, 11)], np.int32),
            np.zeros((0, 2), np.int32),
            np.array([(i, i + 1) for i in range(0, 199, 7)], np.int32),
            np.array([(0, 1), (2, 3), (7, 9)], np.int32),
            workloads.Trajectory(er, 5).next_batch(drsf.DELETE, 400)]
    try:
        for op, per in ((drsf.INSERT, ins), (drsf.DELETE, dels)):
            ub = dev_tensor(np.concatenate([U.shift(i, b) for i, b in enumerate(per)]).reshape(-1, 2))
            vo, bo = _offsets(U, per)
            fp.apply_batched(op, ub, vo, bo)
            got = U.split(fp.parent().cpu().numpy())
            labs = U.split(fp.labels().cpu().numpy())
            for i, g in enumerate(graphs):
                r = oracle.apply(g.n, keys[i], pars[i], op, per[i], want_keys=True)
                assert np.array_equal(got[i], r.parent), (op, i)
                assert np.array_equal(labs[i], oracle.labels(g.n, r.keys)), (op, i)
                keys[i], pars[i] = r.keys, r.parent
    finally:
        fp.close()


def test_persistent_rejects_an_edge_between_graphs():
    """A batch edge with ends in two graphs would merge them: the call is
    skipped and DRSF_EINVAL reported; the handle keeps working."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    graphs = workloads.batched_graphs(4, seed=45, n_lo=500, n_hi=2000)
    U = workloads.Union(graphs)
    fp = drsf.DynamicForest(U.n, dev_tensor(workloads.keys_to_edges(U.keys)), dev_tensor(U.parent))
    try:
        before = fp.parent().cpu().numpy()
        per = [np.array([(0, 1)], np.int32) for _ in graphs]
        bad = np.concatenate([U.shift(i, b) for i, b in enumerate(per)])
        bad[0, 1] = U.offsets[1] + 2          # graph 0's edge reaches into graph 1
        vo, bo = _offsets(U, per)
        fp.apply_batched(drsf.INSERT, dev_tensor(bad), vo, bo)
        with pytest.raises(drsf.DRSFError) as e:
            fp.stats()
        assert e.value.status == drsf.EINVAL
        assert np.array_equal(fp.parent().cpu().numpy(), before)
        tr = workloads.Trajectory(graphs[2], 7)
        b2 = tr.next_batch(drsf.INSERT, 50)
        per = [np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32), b2, np.zeros((0, 2), np.int32)]
        vo, bo = _offsets(U, per)
        fp.apply_batched(drsf.INSERT, dev_tensor(U.shift(2, b2)), vo, bo)
        got = U.split(fp.parent().cpu().numpy())[2]
        r = oracle.apply(graphs[2].n, graphs[2].keys, graphs[2].parent, drsf.INSERT, b2)
        assert np.array_equal(got, r.parent)
    finally:
        fp.close()
