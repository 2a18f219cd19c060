"""Pins of the oracle's batch update (Algorithm 1) on the CPU.

The expected forest F' is derived without the oracle (tests/refs.py): the cut
rule gives F^, networkx gives its pieces, the minimum spanning forest of the
piece graph (scipy, and exhaustive search on tiny inputs) gives E_r, and a
networkx BFS from the smallest piece root of each component of G' orients the
result.  These readings fix F' uniquely, so the comparison is exact.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import refs

nx = pytest.importorskip("networkx")


def _random_case(rng, n, m, op, b):
    keys = workloads.er(n, m, int(rng.integers(1 << 40))) if m else np.zeros(0, np.uint64)
    par = refs.random_forest(n, keys, rng)
    batch = []
    kl = [int(k) for k in keys]
    for _ in range(b):
        r = rng.random()
        if r < 0.1:
            u = int(rng.integers(n))
            batch.append((u, u))                       # self-loop
        elif op == 1 and kl and r < 0.8:
            u, v = refs.ends(kl[rng.integers(len(kl))])  # existing edge
            batch.append((u, v) if rng.random() < 0.5 else (v, u))
        elif op == 1 and kl and r < 0.9:
            v = int(rng.integers(n))
            if par[v] != v:
                batch.append((v, int(par[v])) if rng.random() < 0.5 else (int(par[v]), v))
        else:
            batch.append((int(rng.integers(n)), int(rng.integers(n))))
    if batch and rng.random() < 0.5:
        batch.append(batch[0])                         # duplicate
    return keys, par, np.array(batch, np.int32).reshape(-1, 2)


def _compare(n, keys, par, op, batch, msf=refs.msf_scipy):
    res = oracle.apply(n, keys, par, op, batch, want_keys=True)
    want, er, g2, k, ncross = refs.expected_update(n, keys, par, op, batch, msf=msf)
    assert res.stats["cross"] == ncross
    assert np.array_equal(res.keys, np.array(g2, np.uint64))
    assert [int(x) for x in res.replacement] == er
    assert np.array_equal(res.parent, want), (par, batch, res.parent, want)
    assert oracle.check_forest(n, res.keys, res.parent) == 0
    l = len(set(oracle.labels(n, res.keys).tolist()))
    # Theorem 1: |E_r| = k - l and F' has exactly l roots
    assert res.stats["pieces"] == k and res.stats["components"] == l
    assert len(er) == k - l
    assert int((res.parent == np.arange(n)).sum()) == l
    return res


@pytest.mark.parametrize("op", [0, 1])
def test_tiny_exhaustive_msf(op):
    rng = np.random.default_rng(100 + op)
    for _ in range(150):
        n = int(rng.integers(1, 7))
        m = int(rng.integers(0, n * (n - 1) // 2 + 1))
        keys, par, batch = _random_case(rng, n, m, op, int(rng.integers(0, 5)))
        _compare(n, keys, par, op, batch, msf=refs.msf_bruteforce)


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("n,m,b", [(30, 40, 10), (200, 150, 60), (1000, 1500, 400), (3000, 2500, 1500)])
def test_random_vs_independent(op, n, m, b):
    rng = np.random.default_rng(n * 7 + op)
    for _ in range(3):
        keys, par, batch = _random_case(rng, n, m, op, b)
        _compare(n, keys, par, op, batch)


def test_chain_reversal_closed_form():
    """Cycle 0..n-1, F = path rooted at 0 (parent[i] = i-1).  Deleting tree
    edge {0,1} leaves the single cross edge {0, n-1}; piece {1..n-1} is
    re-rooted at n-1 and hung below 0: parent[i] = i+1 (1 <= i < n-1),
    parent[n-1] = 0.  A linked-list reversal."""
    for n in [3, 4, 10, 1000]:
        keys = np.array(sorted(refs.key(i, (i + 1) % n) for i in range(n)), np.uint64)
        par = np.array([0] + list(range(n - 1)), np.int32)
        res = oracle.apply(n, keys, par, 1, np.array([[1, 0]], np.int32))
        want = np.array([0] + list(range(2, n)) + [0], np.int32)
        assert np.array_equal(res.parent, want)
        assert res.stats["reversed"] == n - 2


def test_insert_into_edgeless_is_kruskal():
    """All-singleton forest: E_r is the minimum spanning forest of B alone and
    each tree is rooted at its smallest vertex."""
    rng = np.random.default_rng(9)
    for n, b in [(2, 1), (50, 80), (2000, 3000)]:
        par = np.arange(n, dtype=np.int32)
        batch = rng.integers(0, n, (b, 2)).astype(np.int32)
        res = oracle.apply(n, np.zeros(0, np.uint64), par, 0, batch, want_keys=True)
        bk = sorted(set(refs.key(u, v) for u, v in batch if u != v))
        er = refs.msf_scipy(n, [(*refs.ends(k), k) for k in bk])
        assert [int(x) for x in res.replacement] == sorted(er)
        T = nx.Graph()
        T.add_nodes_from(range(n))
        T.add_edges_from(refs.ends(k) for k in er)
        want = np.empty(n, np.int32)
        for comp in nx.connected_components(T):
            r = min(comp)
            want[r] = r
            for a, c in nx.bfs_edges(T, r):
                want[c] = a
        assert np.array_equal(res.parent, want)


def test_non_tree_delete_and_internal_insert_keep_forest():
    g = workloads.er_graph(500, 900, seed=4)
    par = g.parent
    nontree = [(u, v) for u, v in g.edges() if par[u] != v and par[v] != u][:50]
    res = oracle.apply(g.n, g.keys, par, 1, np.array(nontree, np.int32))
    assert np.array_equal(res.parent, par) and res.stats["tree_cut"] == 0
    rep = oracle.representatives(par)
    inside = []
    for u in range(g.n):
        for v in range(u + 1, g.n):
            if rep[u] == rep[v] and refs.key(u, v) not in set(g.keys.tolist()):
                inside.append((u, v))
            if len(inside) >= 40:
                break
        if len(inside) >= 40:
            break
    res = oracle.apply(g.n, g.keys, par, 0, np.array(inside, np.int32))
    assert np.array_equal(res.parent, par) and res.stats["replacement"] == 0


def test_normalisation_counts():
    n = 6
    keys = np.array([refs.key(0, 1), refs.key(1, 2)], np.uint64)
    par = np.array([0, 0, 1, 3, 4, 5], np.int32)
    batch = np.array([[3, 3], [0, 1], [3, 4], [4, 3], [2, 5]], np.int32)
    r = oracle.apply(n, keys, par, 0, batch).stats
    assert (r["self_loops"], r["duplicates"], r["ignored"], r["applied"]) == (1, 1, 1, 2)
    r = oracle.apply(n, keys, par, 1, batch).stats
    assert (r["self_loops"], r["duplicates"], r["ignored"], r["applied"]) == (1, 1, 2, 1)
    with pytest.raises(ValueError):
        oracle.apply(n, keys, par, 0, np.array([[0, 6]], np.int32))
    with pytest.raises(ValueError):
        oracle.apply(n, keys, par, 0, np.array([[-1, 2]], np.int32))


def test_trajectory_labels_history_independent():
    """Labels after any batch sequence equal the components of the final G'."""
    g = workloads.rmat_graph(10, 8, seed=21)
    tr = workloads.Trajectory(g, seed=3)
    keys, par = g.keys, g.parent
    for step in range(8):
        op = step % 2
        batch = tr.next_batch(op, 300)
        res = oracle.apply(g.n, keys, par, op, batch, want_keys=True)
        assert np.array_equal(res.keys, workloads.apply_keys(keys, batch, op))
        assert oracle.check_forest(g.n, res.keys, res.parent) == 0
        keys, par = res.keys, res.parent
        tr.advance(batch, op, par)
    lab_oracle = oracle.labels(g.n, keys)
    rep = oracle.representatives(par)
    # every tree of F' is one component; its label is its smallest vertex
    mins = np.full(g.n, g.n, np.int64)
    np.minimum.at(mins, rep, np.arange(g.n))
    assert np.array_equal(mins[rep].astype(np.int32), lab_oracle)
