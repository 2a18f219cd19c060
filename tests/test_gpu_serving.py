"""Serving loop (continuous batching): requests of several tenants overlap
on the device, are coalesced per tenant and admitted under a memory budget.
Each tenant's result in the mix must equal its result alone (its applied
batch log replayed on a fresh handle) and the oracle's."""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_20211_gb300 as drsf
import workloads
from paper_2607_20211_gb300 import serve

pytestmark = pytest.mark.gpu


def _tenants(k, seed):
    out = {}
    for i in range(k):
        g = workloads.er_graph(3000 + 500 * i, 4000 + 700 * i, seed=seed + i) if i % 2 == 0 else \
            workloads.rmat_graph(11 + (i % 3), 8, seed=seed + i)
        out[i] = g
    return out


def _trace(graphs, per_tenant, seed, spread):
    """Requests per tenant (alternating insert / delete batches generated on
    the tenant's oracle trajectory), random arrivals within `spread` s."""
    rng = np.random.default_rng(seed)
    reqs = []
    rid = 0
    for tid, g in graphs.items():
        tr = workloads.Trajectory(g, seed=seed * 100 + tid)
        keys, par = g.keys, g.parent
        times = np.sort(rng.uniform(0, spread, per_tenant))
        for j in range(per_tenant):
            op = int(rng.random() < 0.4)
            b = int(rng.integers(50, 600))
            batch = tr.next_batch(op, b)
            r = oracle.apply(g.n, keys, par, op, batch, want_keys=True)
            keys, par = r.keys, r.parent
            tr.advance(batch, op, par)
            reqs.append(serve.Request(rid, tid, op, batch, float(times[j])))
            rid += 1
    return reqs


def _replay_alone(g, log):
    keys, par = g.keys, g.parent
    f = drsf.DynamicForest(g.n, torch.from_numpy(g.edges()).cuda(), torch.from_numpy(g.parent).cuda())
    for op, b in log:
        f.apply_host(op, b)
        keys = oracle.apply(g.n, keys, par, op, b, want_keys=True)
        par = keys.parent
        keys = keys.keys
    out = f.parent().cpu().numpy()
    f.close()
    return out, par


@pytest.mark.parametrize("coalesce,budget", [(True, 120 << 30), (False, 120 << 30), (True, 20 << 20)])
def test_mix_equals_alone(coalesce, budget):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    graphs = _tenants(6, seed=70)
    reqs = _trace(graphs, per_tenant=8, seed=71, spread=0.002)
    s = serve.Server(budget_bytes=budget, slots=4, coalesce=coalesce)
    for tid, g in graphs.items():
        s.add_tenant(tid, g.n, g.edges(), g.parent)
    done = s.run(reqs)
    assert sorted(d.rid for d in done) == sorted(r.rid for r in reqs)
    for tid, g in graphs.items():
        _, par_mix = s.state(tid)
        alone_gpu, alone_oracle = _replay_alone(g, s.tenants[tid].log)
        assert np.array_equal(par_mix, alone_gpu), tid
        assert np.array_equal(par_mix, alone_oracle), tid
        if not coalesce:
            assert len(s.tenants[tid].log) == sum(1 for r in reqs if r.tenant == tid)
    if budget < (1 << 30):
        assert s.evictions > 0
    stats = serve.summarize(done)
    assert stats["requests"] == len(reqs)


def test_coalesced_mix_keeps_labels_and_validity_per_request_sequence():
    """With coalescing, a tenant's forest in the mix is its coalesced log
    replayed alone (tested above); against its original request sequence
    applied one by one, the labels must be identical and the mix's forest
    must be a valid rooted spanning forest of the same graph (a merged batch
    may pick other replacement edges, so the parent arrays may differ)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    drsf.build()
    graphs = _tenants(4, seed=80)
    reqs = _trace(graphs, per_tenant=10, seed=81, spread=0.001)
    s = serve.Server(budget_bytes=120 << 30, slots=4, coalesce=True)
    for tid, g in graphs.items():
        s.add_tenant(tid, g.n, g.edges(), g.parent)
    s.run(reqs)
    for tid, g in graphs.items():
        keys, par = g.keys, g.parent
        for r in sorted((r for r in reqs if r.tenant == tid), key=lambda r: (r.t_arrive, r.rid)):
            o = oracle.apply(g.n, keys, par, r.op, r.batch, want_keys=True)
            keys, par = o.keys, o.parent
        _, par_mix = s.state(tid)
        assert oracle.check_forest(g.n, keys, par_mix) == 0, tid
        lab_mix = oracle.labels(g.n, keys)
        # labels from the mix's own forest: the smallest vertex id of each tree
        v = np.arange(g.n)
        roots = par_mix.copy()
        for _ in range(40):   # pointer doubling: depth up to 2^40
            roots = roots[roots]
        mins = np.full(g.n, g.n, np.int64)
        np.minimum.at(mins, roots, v)
        assert np.array_equal(mins[roots], lab_mix), tid
    s.close()
