"""Independent expectations used to pin the oracle (test side only).

Nothing here calls the oracle.  Each routine derives the expected result
another way: brute-force enumeration on tiny inputs, or a library routine
(scipy's minimum spanning tree, networkx's BFS) for a special case the paper's
definitions reduce to.
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np


def key(u, v):
    u, v = int(u), int(v)
    return (min(u, v) << 32) | max(u, v)


def ends(k):
    k = int(k)
    return k >> 32, k & 0xFFFFFFFF


def components(n, edges):
    """Component id (smallest vertex) per vertex, by BFS over python lists."""
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    lab = [-1] * n
    for s in range(n):
        if lab[s] != -1:
            continue
        lab[s] = s
        dq = deque([s])
        while dq:
            x = dq.popleft()
            for y in adj[x]:
                if lab[y] == -1:
                    lab[y] = s
                    dq.append(y)
    return lab


def rooted_forests(n, edges):
    """Every rooted spanning forest of the graph (n, edges), as parent tuples.

    Enumerates edge subsets of size n - c(G) that are acyclic (hence spanning
    forests), then every choice of one root per tree, orienting edges towards
    the root."""
    lab = components(n, edges)
    c = len(set(lab))
    need = n - c
    out = set()
    for sub in itertools.combinations(range(len(edges)), need):
        uf = list(range(n))

        def f(x):
            while uf[x] != x:
                x = uf[x]
            return x
        ok = True
        for i in sub:
            a, b = f(edges[i][0]), f(edges[i][1])
            if a == b:
                ok = False
                break
            uf[a] = b
        if not ok:
            continue
        tl = components(n, [edges[i] for i in sub])
        trees = {}
        for v in range(n):
            trees.setdefault(tl[v], []).append(v)
        tadj = [[] for _ in range(n)]
        for i in sub:
            u, v = edges[i]
            tadj[u].append(v)
            tadj[v].append(u)
        for roots in itertools.product(*trees.values()):
            par = [-1] * n
            for r in roots:
                par[r] = r
                dq = deque([r])
                while dq:
                    x = dq.popleft()
                    for y in tadj[x]:
                        if par[y] == -1:
                            par[y] = x
                            dq.append(y)
            out.add(tuple(par))
    return out


def normalise(keys, op, batch):
    """Batch normalisation reading: the set of applied keys and G'."""
    G = set(int(k) for k in keys)
    seen, applied = set(), []
    for u, v in np.asarray(batch).reshape(-1, 2):
        if u == v:
            continue
        k = key(u, v)
        if k in seen:
            continue
        seen.add(k)
        if (op == 0) == (k in G):
            continue
        applied.append(k)
    G2 = G | set(applied) if op == 0 else G - set(applied)
    return applied, G2


def msf_scipy(n_pieces, pedges):
    """Minimum spanning forest of a multigraph on pieces 0..n_pieces-1 whose
    edges are (piece_a, piece_b, key); weights are key ranks (distinct).
    Uses scipy.sparse.csgraph.minimum_spanning_tree.  Returns the set of keys."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    best = {}
    for a, b, k in pedges:
        p = (min(a, b), max(a, b))
        if p not in best or k < best[p]:
            best[p] = k
    if not best:
        return set()
    items = sorted(best.items(), key=lambda t: t[1])
    rows = [p[0] for p, _ in items]
    cols = [p[1] for p, _ in items]
    w = np.arange(1, len(items) + 1, dtype=np.float64)
    M = coo_matrix((w, (rows, cols)), shape=(n_pieces, n_pieces)).tocsr()
    T = minimum_spanning_tree(M).tocoo()
    by_pair = {p: k for p, k in items}
    return {by_pair[(min(int(r), int(c)), max(int(r), int(c)))] for r, c in zip(T.row, T.col)}


def msf_bruteforce(n_pieces, pedges):
    """Same as msf_scipy by exhaustive search: among acyclic edge subsets of
    maximum size, the one with the smallest sum of key ranks."""
    ks = sorted(set(k for _, _, k in pedges))
    rank = {k: i for i, k in enumerate(ks)}
    e = [(a, b, k) for a, b, k in pedges]
    bestset, bestsize, bestw = set(), -1, None
    for r in range(len(e), -1, -1):
        if r < bestsize:
            break
        for sub in itertools.combinations(e, r):
            uf = list(range(n_pieces))

            def f(x):
                while uf[x] != x:
                    x = uf[x]
                return x
            ok = True
            for a, b, _ in sub:
                x, y = f(a), f(b)
                if x == y:
                    ok = False
                    break
                uf[x] = y
            if not ok:
                continue
            w = sum(rank[k] for _, _, k in sub)
            if r > bestsize or w < bestw:
                bestset, bestsize, bestw = {k for _, _, k in sub}, r, w
    return bestset


def expected_update(n, keys, parent, op, batch, msf=msf_scipy):
    """The unique F' fixed by the deterministic readings, derived without the
    oracle: F^ by the cut rule, pieces by networkx components, E_r as the
    minimum spanning forest of the piece graph, roots = smallest piece root per
    component of G', orientation by networkx BFS from those roots."""
    import networkx as nx
    applied, G2 = normalise(keys, op, batch)
    par = [int(p) for p in parent]
    if op == 1:
        for k in applied:
            a, c = ends(k)
            if par[a] == c:
                par[a] = a
            elif par[c] == a:
                par[c] = c
    F = nx.Graph()
    F.add_nodes_from(range(n))
    F.add_edges_from((v, par[v]) for v in range(n) if par[v] != v)
    piece_of = {}
    proot = []
    for i, comp in enumerate(nx.connected_components(F)):
        roots = [v for v in comp if par[v] == v]
        assert len(roots) == 1
        proot.append(roots[0])
        for v in comp:
            piece_of[v] = i
    pedges = []
    for k in G2:
        a, c = ends(k)
        if piece_of[a] != piece_of[c]:
            pedges.append((piece_of[a], piece_of[c], k))
    er = msf(len(proot), pedges)
    T = nx.Graph()
    T.add_nodes_from(range(n))
    T.add_edges_from((v, par[v]) for v in range(n) if par[v] != v)
    T.add_edges_from(ends(k) for k in er)
    out = [-1] * n
    for comp in nx.connected_components(T):
        r = min(proot[piece_of[v]] for v in comp)
        out[r] = r
        for a, b in nx.bfs_edges(T, r):
            out[b] = a
    return np.array(out, np.int32), sorted(er), sorted(G2), len(proot), len(pedges)


def random_forest(n, keys, rng):
    """A random rooted spanning forest of (n, keys): random-order Kruskal
    spanning forest, random root per tree, networkx BFS orientation."""
    import networkx as nx
    ks = list(int(k) for k in keys)
    rng.shuffle(ks)
    uf = list(range(n))

    def f(x):
        while uf[x] != x:
            uf[x] = uf[uf[x]]
            x = uf[x]
        return x
    T = nx.Graph()
    T.add_nodes_from(range(n))
    for k in ks:
        a, c = ends(k)
        x, y = f(a), f(c)
        if x != y:
            uf[x] = y
            T.add_edge(a, c)
    par = np.empty(n, np.int32)
    for comp in nx.connected_components(T):
        comp = sorted(comp)
        r = comp[rng.integers(len(comp))]
        par[r] = r
        for a, b in nx.bfs_edges(T, r):
            par[b] = a
    return par
