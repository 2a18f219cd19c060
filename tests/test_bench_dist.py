"""Multi-process (gloo, world size 2, CPU) checks of the benchmark's
replica aggregation: whole-job units are summed over ranks and divided by
the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank)
    bench.barrier()
    q.put((rank, units, secs))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, units, secs in res:
        assert units == 3000.0 and secs == 1.5


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)


def test_phase_bytes_model_positive():
    import bench
    st = dict(batch_len=10, applied=8, candidates=5, active=3, affected=20, detached=7, scanned=40, tree_cut=4,
              jump_rounds=3, replacement=2, rank_rounds=2, mark_rounds=2, reversed=1, hook_rounds=2)
    for op in (0, 1):
        by = bench.phase_bytes(st, 100, op)
        assert all(v >= 0 for v in by.values()) and by["begin"] == 80
    # the per-unit figures: 12 per affected vertex and doubling round; 12 per
    # scanned row + 8 per entry + 8 per candidate; 24 per candidate and round
    by = bench.phase_bytes(st, 100, 1)
    assert by["jump"] == 12 * 20 * 3   # no visit count: affected x rounds
    st2 = dict(st, jump_visits=45)
    assert bench.phase_bytes(st2, 100, 1)["jump"] == 12 * 45
    assert by["scan"] == 12 * 7 + 8 * 40 + 8 * 5
    assert by["hook"] == 24 * 5 * 2
    assert by["reverse"] == 12 * 1 + 8 * 2
