"""The pooled trajectory check (tests/oracle_pool.py) on the CPU: a trajectory
produced by the oracle itself passes, and a planted change in one batch's
parent array, labels or counters is reported (so a GPU mismatch cannot slip
through the pool)."""
import numpy as np
import pytest

import oracle
import workloads
from tests.oracle_pool import TrajectoryCheck


def _oracle_trajectory(g, schedule, seed):
    tr = workloads.Trajectory(g, seed)
    keys, par = g.keys, g.parent
    out = []
    for op, b in schedule:
        batch = tr.next_batch(op, b)
        r = oracle.apply(g.n, keys, par, op, batch, want_keys=True)
        st = {"applied": r.stats["applied"], "self_loops": r.stats["self_loops"],
              "dropped": r.stats["duplicates"] + r.stats["ignored"], "tree_cut": r.stats["tree_cut"],
              "replacement": r.stats["replacement"], "edges": r.stats["m_out"]}
        out.append((op, batch, r.parent.copy(), st, oracle.labels(g.n, r.keys)))
        keys, par = r.keys, r.parent
        tr.advance(batch, op, par)
    return out


SCHED = [(0, 300), (1, 300), (0, 300), (1, 300)]


def _run(g, traj):
    chk = TrajectoryCheck(g.n, g.keys, g.parent)
    for op, batch, par, st, lab in traj:
        chk.add(op, batch, par, st, lab)
    return chk.result()


def test_pool_accepts_the_oracle_trajectory():
    g = workloads.er_graph(3000, 3600, seed=7)
    assert _run(g, _oracle_trajectory(g, SCHED, seed=8)) == 4


@pytest.mark.parametrize("what", ["parent", "labels", "counter"])
def test_pool_reports_a_planted_mismatch(what):
    g = workloads.er_graph(3000, 3600, seed=7)
    traj = _oracle_trajectory(g, SCHED, seed=8)
    op, batch, par, st, lab = traj[2]
    if what == "parent":
        par = par.copy()
        v = int(np.nonzero(par != np.arange(g.n))[0][0])
        par[v] = v                      # one extra root
    elif what == "labels":
        lab = lab.copy()
        lab[-1] = (lab[-1] + 1) % g.n
    else:
        st = dict(st, replacement=st["replacement"] + 1)
    traj[2] = (op, batch, par, st, lab)
    with pytest.raises(AssertionError, match="batch 2"):
        _run(g, traj)
