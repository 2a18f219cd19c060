"""GPU parity: the CUDA path against the serial oracle, batch by batch.

Bar: the parent array equals the oracle's bit for bit (deterministic mode:
minimum-key replacement edges, smallest-root super-roots), the labels equal
the oracle's component minima, the exact checker accepts the forest, and the
per-batch counters agree.  Integer work only, so every comparison is exact.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_20211_gb300 as drsf
import workloads
from tests.gpu_util import check_batch, dev_tensor, make_forest, run_trajectory

pytestmark = pytest.mark.gpu

I, D = drsf.INSERT, drsf.DELETE


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()


def test_er_small_config():
    """Erdos-Renyi n=20,000, m=25,000 (seed 1): one insert batch of 2,000 new
    pairs, then one delete batch of 2,000 edges (half tree edges)."""
    g = workloads.er_graph(20_000, 25_000, seed=1)
    run_trajectory(g, [(I, 2000), (D, 2000)], seed=1)


def test_er_multi_batch():
    g = workloads.er_graph(20_000, 25_000, seed=11)
    run_trajectory(g, [(I, 3000), (D, 3000)] * 4, seed=12)


def test_rmat16_trajectory():
    g = workloads.rmat_graph(16, 16, seed=2)
    run_trajectory(g, [(I, 1000), (D, 1000), (I, 10_000), (D, 10_000)] * 3, seed=3)


def test_sparse_rows_scan():
    """Average degree ~2: delete scans cover long runs of one- and two-entry
    rows, so scan tiles span many rows."""
    g = workloads.er_graph(200_000, 200_000, seed=17)
    run_trajectory(g, [(D, 20_000), (I, 20_000)] * 3, seed=18, tree_frac=0.7)


def test_grid_deep_paths():
    """Grid 512 x 512, p = 0.6, deletes with 90% tree edges (long reversals),
    local inserts within 64 cells."""
    g = workloads.grid_graph(512, 512, seed=3)
    st = run_trajectory(g, [(D, 5000), (I, 5000)] * 3, seed=4, tree_frac=0.9, local=64)
    assert st is not None


@pytest.mark.parametrize("variant", ["sync", "halving"])
def test_root_search_variants(variant, monkeypatch):
    """The selectable root searches of delete batches (synchronous doubling
    rounds, path-halving walks) give the oracle's forest too; R-MAT-16 and a
    deep grid (long doubling chains)."""
    monkeypatch.setenv("DRSF_JUMP", variant)
    monkeypatch.setenv("DRSF_DETACH", "0")   # root search for every delete (no top-down search first)
    g = workloads.rmat_graph(16, 16, seed=2)
    run_trajectory(g, [(I, 1000), (D, 1000), (I, 10_000), (D, 10_000)] * 2, seed=3)
    g = workloads.grid_graph(256, 256, seed=3)
    run_trajectory(g, [(D, 2000), (I, 2000)] * 2, seed=4, tree_frac=0.9, local=64)


def test_deterministic_run_to_run():
    g = workloads.rmat_graph(14, 8, seed=5)
    tr = workloads.Trajectory(g, seed=6)
    b1 = tr.next_batch(D, 3000)
    outs = []
    for _ in range(2):
        f = make_forest(g)
        f.apply(D, dev_tensor(b1))
        outs.append(f.parent().cpu().numpy())
        f.close()
    assert np.array_equal(outs[0], outs[1])


def _tiny(n, edges, parent):
    keys = workloads.edges_to_keys(np.array(edges, np.int64).reshape(-1, 2)) if edges else np.zeros(0, np.uint64)
    g = workloads.Graph.__new__(workloads.Graph)
    g.name, g.n, g.keys, g.W = "tiny", n, keys, 0
    g.parent = np.array(parent, np.int32) if parent is not None else workloads.bfs_forest(n, keys)
    return g


def test_edge_cases():
    # n = 1, empty graph, empty batch and a self-loop
    g = _tiny(1, [], [0])
    f = make_forest(g)
    for op, b in [(I, np.zeros((0, 2), np.int32)), (I, np.array([[0, 0]], np.int32)),
                  (D, np.array([[0, 0]], np.int32))]:
        check_batch(f, 1, g.keys, g.parent, op, b)
    f.close()
    # star, then duplicates / existing / absent / self-loops
    n = 50
    g = _tiny(n, [(0, i) for i in range(1, n)], None)
    f = make_forest(g)
    keys, par = g.keys, g.parent
    b = np.array([[3, 3], [1, 2], [2, 1], [0, 5], [7, 9], [9, 7], [9, 7]], np.int32)
    keys, par, st = check_batch(f, n, keys, par, I, b)
    b = np.array([[0, 5], [5, 0], [4, 6], [1, 2], [0, 1], [8, 8]], np.int32)
    keys, par, st = check_batch(f, n, keys, par, D, b)
    # delete every tree edge of the star: all leaves become singletons or re-hang
    b = np.array([[0, i] for i in range(1, n)], np.int32)
    keys, par, st = check_batch(f, n, keys, par, D, b)
    f.close()
    # insert into an edgeless graph (pure Kruskal)
    n = 3000
    g = _tiny(n, [], list(range(n)))
    f = make_forest(g)
    rng = np.random.default_rng(1)
    check_batch(f, n, g.keys, g.parent, I, rng.integers(0, n, (5000, 2)).astype(np.int32))
    f.close()


def test_long_path_reversal():
    """A single path of 200,000 vertices rooted at 0 plus the closing edge;
    deleting the first tree edge re-roots the whole path (depth n - 1)."""
    n = 200_000
    edges = [(i, i + 1) for i in range(n - 1)] + [(0, n - 1)]
    g = _tiny(n, edges, [0] + list(range(n - 1)))
    f = make_forest(g)
    keys, par, st = check_batch(f, n, g.keys, g.parent, D, np.array([[1, 0]], np.int32))
    assert st["reversed"] == n - 2
    # and several cuts at once along the path
    b = np.array([[k, k + 1] for k in range(5000, n - 1, 17_000)], np.int32)
    check_batch(f, n, keys, par, D, b)
    f.close()


def test_walk_length_boundary():
    """Re-rooted paths of 1 .. 130 edges in one batch, around the 64-edge
    limit of the walking reversal (longer paths go through the marks):
    paths hang below their top vertex, vertex 0 is a lone root with the
    smallest id, and one insert joins each path's deepest vertex to 0, so
    every path is re-rooted at its deep end."""
    lengths = [1, 2, 31, 63, 64, 65, 66, 100, 130]
    n = 1 + sum(L + 1 for L in lengths)
    edges, parent = [], [0]
    leaves, tops, v = [], [], 1
    for L in lengths:
        top = v
        parent.append(top)
        for k in range(1, L + 1):
            edges.append((v + k - 1, v + k))
            parent.append(v + k - 1)
        tops.append(top)
        leaves.append(v + L)
        v += L + 1
    g = _tiny(n, edges, parent)
    f = make_forest(g)
    b = np.array([[leaf, 0] for leaf in leaves], np.int32)
    keys, par, st = check_batch(f, n, g.keys, g.parent, I, b)
    assert st["reversed"] == sum(lengths)
    # cut every path in its middle and join the halves back through 0
    b = np.array([[tops[i] + L // 2, tops[i] + L // 2 + 1] for i, L in enumerate(lengths)], np.int32)
    keys, par, st = check_batch(f, n, keys, par, D, b)
    b = np.array([[t, 0] for t in tops], np.int32)
    check_batch(f, n, keys, par, I, b)
    f.close()


def test_invalid_id_skips_batch():
    g = workloads.er_graph(1000, 1500, seed=7)
    f = make_forest(g)
    before = f.parent().cpu().numpy()
    f.apply(I, dev_tensor(np.array([[0, 1], [2, 1000]], np.int32)))
    with pytest.raises(drsf.DRSFError) as e:
        f.sync()
    assert e.value.status == drsf.EINVAL
    assert np.array_equal(f.parent().cpu().numpy(), before)
    assert f.num_edges() == g.m
    # the handle stays usable
    tr = workloads.Trajectory(g, seed=8)
    check_batch(f, g.n, g.keys, g.parent, I, tr.next_batch(I, 100))
    f.close()


def test_apply_host_matches_device():
    g = workloads.rmat_graph(14, 8, seed=9)
    tr = workloads.Trajectory(g, seed=10)
    b = tr.next_batch(D, 2000)
    f1, f2 = make_forest(g), make_forest(g)
    f1.apply(D, dev_tensor(b))
    f2.apply_host(D, b)
    assert np.array_equal(f1.parent().cpu().numpy(), f2.parent().cpu().numpy())
    f1.close()
    f2.close()


def test_overflow_and_rebuild():
    """Rows fill past their slack (edges spill to the overflow list) and the
    index fills past its load limit (storage rebuild), with parity kept."""
    g = workloads.er_graph(4000, 4000, seed=13)
    st = run_trajectory(g, [(I, 60_000)] * 4 + [(D, 30_000), (I, 40_000), (D, 50_000)], seed=14,
                        labels=True)
    assert st["rebuilds"] >= 1


def test_validate_flag():
    g = workloads.er_graph(500, 800, seed=15)
    f = make_forest(g, flags=drsf.DETERMINISTIC | drsf.VALIDATE)
    f.close()
    bad = g.parent.copy()
    roots = np.nonzero(bad == np.arange(g.n))[0]
    # give a root a parent that is not its neighbour
    r = int(roots[0])
    bad[r] = (r + 1) % g.n if (r + 1) % g.n != r else r
    with pytest.raises(drsf.DRSFError) as e:
        drsf.DynamicForest(g.n, dev_tensor(g.edges()), dev_tensor(bad), flags=drsf.VALIDATE)
    assert e.value.status in (drsf.ENOT_FOREST,)


@pytest.mark.parametrize("variant", ["sg", "hs"])
def test_replacement_edge_variants(variant):
    """Both replacement-edge variants of Section III, forced for every batch:
    the supergraph reduction (one minimum-key edge per pair of trees) and
    hooking on every cross edge give the oracle's forest bit for bit, on
    inserts and deletes alike."""
    flags = drsf.DETERMINISTIC | (drsf.REPL_SG if variant == "sg" else drsf.REPL_HS)
    g = workloads.er_graph(20_000, 25_000, seed=1)
    st = run_trajectory(g, [(I, 2000), (D, 2000)] * 2, seed=1, flags=flags)
    assert st["supergraph"] == (1 if variant == "sg" else 0)
    g = workloads.rmat_graph(16, 16, seed=2)
    run_trajectory(g, [(I, 1000), (D, 1000), (I, 10_000), (D, 10_000)] * 2, seed=3, flags=flags)
    g = workloads.grid_graph(512, 512, seed=3)
    run_trajectory(g, [(D, 5000), (I, 5000)] * 2, seed=4, tree_frac=0.9, local=64, flags=flags)


def test_direct_launches_without_captured_graphs(monkeypatch):
    """Batches are replayed from captured CUDA graphs by default; with
    DRSF_GRAPHS=0 every kernel is launched one by one.  Both give the
    oracle's forests (R-MAT-16 trajectory with a storage rebuild forced by
    growth, which moves the storage the captured graphs point into)."""
    g = workloads.rmat_graph(16, 16, seed=2)
    for env in ("0", "1"):
        monkeypatch.setenv("DRSF_GRAPHS", env)
        run_trajectory(g, [(I, 1000), (D, 1000), (I, 60_000), (D, 10_000), (I, 200_000), (D, 50_000)], seed=3)


def test_top_down_detach_and_its_fallback(monkeypatch):
    """Deletes look for their detached vertices top-down from the cut
    vertices first and hand over to pointer jumping when that search runs
    over its budget (here: the level limit on a deep grid).  Both paths give
    the oracle's forests; the counters show which one each batch took; and
    with DRSF_DETACH=0 the same trajectories match too."""
    seen = {"top": 0, "fallback": 0}

    def watch(g, schedule, seed, **kw):
        f = make_forest(g)
        keys, par = g.keys, g.parent
        tr = workloads.Trajectory(g, seed, tree_frac=kw.get("tree_frac", 0.5), local=kw.get("local", 0))
        try:
            for op, b in schedule:
                batch = tr.next_batch(op, b)
                keys, par, st = check_batch(f, g.n, keys, par, op, batch)
                tr.advance(batch, op, par)
                if op == D and st["tree_cut"] > 0:
                    seen["top" if st["detach_levels"] > 0 else "fallback"] += 1
        finally:
            f.close()

    watch(workloads.rmat_graph(16, 16, seed=2), [(I, 1000), (D, 1000), (I, 10_000), (D, 10_000)] * 2, seed=3)
    watch(workloads.grid_graph(1024, 1024, seed=3), [(D, 20_000), (I, 20_000)] * 2, seed=4, tree_frac=0.9,
          local=64)
    assert seen["top"] > 0 and seen["fallback"] > 0, seen
    monkeypatch.setenv("DRSF_DETACH", "0")
    run_trajectory(workloads.rmat_graph(16, 16, seed=2), [(I, 1000), (D, 1000), (I, 10_000), (D, 10_000)], seed=3)


def test_top_down_level_limit_skip_and_retry():
    """A path of 20,000 vertices rooted at 0: every cut detaches a chain far
    deeper than the top-down search's level limit (16), and small enough for
    its vertex and entry budgets, so the search gives up at the limit
    (detach_levels == -16), the next 8 deletes skip it (detach_levels == 0:
    pointer jumping from the start), and the one after tries it again.
    Every batch matches the oracle."""
    n = 20_000
    edges = [(i, i + 1) for i in range(n - 1)]
    g = _tiny(n, edges, [0] + list(range(n - 1)))
    f = make_forest(g)
    keys, par = g.keys, g.parent
    levels = []
    try:
        for b in range(10):
            k = 100 * (b + 1)
            keys, par, st = check_batch(f, n, keys, par, D, np.array([[k, k + 1]], np.int32))
            assert st["tree_cut"] == 1
            levels.append(st["detach_levels"])
    finally:
        f.close()
    assert levels == [-16] + [0] * 8 + [-16], levels
