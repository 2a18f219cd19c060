"""Shared helpers of the GPU parity tests: drive the CUDA library and the
serial oracle through the same seeded trajectory and compare every batch."""
import numpy as np
import torch

import oracle
import paper_2607_20211_gb300 as drsf
import workloads


def dev_tensor(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def make_forest(g, flags=drsf.DETERMINISTIC):
    return drsf.DynamicForest(g.n, dev_tensor(g.edges().reshape(-1, 2)), dev_tensor(g.parent), flags=flags)


def check_batch(f, n, keys, par, op, batch, labels=True):
    """Apply `batch` on the GPU and compare with the oracle; return the
    oracle's (keys', parent')."""
    f.apply(op, dev_tensor(batch.reshape(-1, 2)))
    got = f.parent().cpu().numpy()
    st = f.stats()
    ref = oracle.apply(n, keys, par, op, batch, want_keys=True)
    if not np.array_equal(got, ref.parent):
        bad = np.nonzero(got != ref.parent)[0]
        raise AssertionError(f"parent differs at {len(bad)} vertices, first {bad[:10].tolist()}: "
                             f"gpu {got[bad[:10]].tolist()} oracle {ref.parent[bad[:10]].tolist()}; "
                             f"gpu stats {st} oracle stats {ref.stats}")
    assert oracle.check_forest(n, ref.keys, got) == 0
    assert st["applied"] == ref.stats["applied"]
    assert st["self_loops"] == ref.stats["self_loops"]
    assert st["dropped"] == ref.stats["duplicates"] + ref.stats["ignored"]
    assert st["tree_cut"] == ref.stats["tree_cut"]
    assert st["replacement"] == ref.stats["replacement"], (st, ref.stats)
    assert st["edges"] == ref.stats["m_out"]
    if labels:
        lab = f.labels().cpu().numpy()
        assert np.array_equal(lab, oracle.labels(n, ref.keys))
    return ref.keys, ref.parent, st


def run_trajectory(g, schedule, seed, tree_frac=0.5, local=0, labels=True, flags=drsf.DETERMINISTIC):
    """schedule: list of (op, batch size).  Returns the last GPU stats."""
    f = make_forest(g, flags=flags)
    keys, par = g.keys, g.parent
    tr = workloads.Trajectory(g, seed, tree_frac=tree_frac, local=local)
    st = None
    try:
        for op, b in schedule:
            batch = tr.next_batch(op, b)
            keys, par, st = check_batch(f, g.n, keys, par, op, batch, labels=labels)
            tr.advance(batch, op, par)
    finally:
        f.close()
    return st


def _tiny_graph(n, edges, parent):
    """A Graph from an explicit edge list and parent array (None: BFS forest)."""
    keys = workloads.edges_to_keys(np.array(edges, np.int64).reshape(-1, 2)) if edges else np.zeros(0, np.uint64)
    g = workloads.Graph.__new__(workloads.Graph)
    g.name, g.n, g.keys, g.W = "tiny", n, keys, 0
    g.parent = np.array(parent, np.int32) if parent is not None else workloads.bfs_forest(n, keys)
    return g


def run_trajectory_pooled(g, schedule, seed, tree_frac=0.5, local=0, labels=True, flags=drsf.DETERMINISTIC):
    """As run_trajectory, for long or large trajectories: the GPU runs the
    whole schedule and every batch is checked against the oracle in the
    process pool of tests/oracle_pool.py (same checks, side by side).
    Returns the number of batches checked."""
    from tests.oracle_pool import TrajectoryCheck
    chk = TrajectoryCheck(g.n, g.keys, g.parent)
    f = make_forest(g, flags=flags)
    tr = workloads.Trajectory(g, seed, tree_frac=tree_frac, local=local)
    try:
        for op, b in schedule:
            batch = tr.next_batch(op, b)
            f.apply(op, dev_tensor(batch.reshape(-1, 2)))
            par = f.parent().cpu().numpy()
            st = f.stats()
            lab = f.labels().cpu().numpy() if labels else None
            chk.add(op, batch, par, st, lab)
            tr.advance(batch, op, par)
    finally:
        f.close()
    return chk.result()
