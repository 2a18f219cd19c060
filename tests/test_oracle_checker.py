"""Pins of the oracle's exact forest checker and labels (CPU only).

The checker (D-RSF box, Section I; rooted spanning forest, Section II-A) is
compared with brute-force enumeration of every rooted spanning forest on all
graphs with n <= 4 and a sample of graphs with n = 5, over every parent array.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests import refs


def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


def _check_graph(n, edges):
    keys = np.array(sorted(refs.key(u, v) for u, v in edges), np.uint64)
    valid = refs.rooted_forests(n, edges)
    assert valid, "every graph has a rooted spanning forest"
    for par in itertools.product(range(n), repeat=n):
        got = oracle.check_forest(n, keys, np.array(par, np.int32))
        assert (got == 0) == (par in valid), (n, edges, par, got)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_checker_exhaustive(n):
    for edges in _all_graphs(n):
        _check_graph(n, edges)


def test_checker_n5_sample():
    rng = np.random.default_rng(11)
    graphs = list(_all_graphs(5))
    for i in rng.choice(len(graphs), 150, replace=False):
        _check_graph(5, graphs[i])


def test_checker_failure_codes():
    # path 0-1-2-3 plus edge 0-3; n = 4
    keys = np.array(sorted(refs.key(*e) for e in [(0, 1), (1, 2), (2, 3), (0, 3)]), np.uint64)
    ok = np.array([0, 0, 1, 2], np.int32)
    assert oracle.check_forest(4, keys, ok) == oracle.CHECK_OK
    assert oracle.check_forest(4, keys, np.array([0, 0, 1, 7], np.int32)) == oracle.CHECK_RANGE
    assert oracle.check_forest(4, keys, np.array([0, 0, 0, 2], np.int32)) == oracle.CHECK_NOT_EDGE
    assert oracle.check_forest(4, keys, np.array([1, 2, 3, 0], np.int32)) == oracle.CHECK_CYCLE
    assert oracle.check_forest(4, keys, np.array([0, 0, 2, 2], np.int32)) == oracle.CHECK_ROOTS
    # two components, one without a root: 0-1 and 2-3 (2 <-> 3 cycle is rule 3)
    keys2 = np.array([refs.key(0, 1), refs.key(2, 3)], np.uint64)
    assert oracle.check_forest(4, keys2, np.array([0, 0, 3, 2], np.int32)) == oracle.CHECK_CYCLE
    assert oracle.check_forest(4, keys2, np.array([0, 0, 2, 3], np.int32)) == oracle.CHECK_ROOTS


def test_labels_vs_scipy():
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(5)
    for n, m in [(1, 0), (10, 0), (50, 30), (2000, 1500), (5000, 20000)]:
        u = rng.integers(0, n, m)
        v = rng.integers(0, n, m)
        keep = u != v
        keys = np.unique((np.minimum(u, v)[keep].astype(np.uint64) << np.uint64(32))
                         | np.maximum(u, v)[keep].astype(np.uint64))
        a = (keys >> np.uint64(32)).astype(np.int64)
        b = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
        M = coo_matrix((np.ones(len(keys)), (a, b)), shape=(n, n))
        nc, lab = connected_components(M, directed=False)
        mins = np.full(nc, n, np.int64)
        np.minimum.at(mins, lab, np.arange(n))
        assert np.array_equal(oracle.labels(n, keys), mins[lab].astype(np.int32))


def test_representatives_known_roots():
    import networkx as nx
    rng = np.random.default_rng(3)
    for n in [1, 7, 300]:
        T = nx.random_labeled_tree(n, seed=int(rng.integers(1 << 30))) if n > 1 else nx.empty_graph(1)
        # split into a forest by dropping some edges, root each tree at a chosen vertex
        es = list(T.edges())
        drop = set(rng.choice(len(es), len(es) // 3, replace=False).tolist()) if es else set()
        F = nx.Graph()
        F.add_nodes_from(range(n))
        F.add_edges_from(e for i, e in enumerate(es) if i not in drop)
        par = np.empty(n, np.int32)
        want = np.empty(n, np.int32)
        for comp in nx.connected_components(F):
            comp = sorted(comp)
            r = comp[len(comp) // 2]
            par[r] = r
            for a, b in nx.bfs_edges(F, r):
                par[b] = a
            want[comp] = r
        assert np.array_equal(oracle.representatives(par), want)
    with pytest.raises(ValueError):
        oracle.representatives(np.array([1, 0], np.int32))
