"""Host logic of the batched form's autotuner (CPU): coordinate descent picks
the fastest candidate per size class and operation, the cache round-trips,
and a different workload signature does not reuse it.  The timing function is
replaced by a synthetic cost model; no GPU is touched."""
import numpy as np

from paper_2607_20211_gb300 import DEFAULT_CLASSES, autotune


def test_tune_picks_the_fastest_schedule_and_caches_it(tmp_path, monkeypatch):
    best = {0: {0: (512, 0, 1), 1: (1024, 0, 2), 2: (1024, 0, 8)}, 1: {0: (256, 0, 2), 1: (1024, 1, 1), 2: (1024, 0, 16)}}

    def fake_time(n, edges, parent, op, batch, vo, bo, classes):
        # each class costs 1 ms, 0.1 ms when it runs its preferred schedule
        return sum(0.1 if tuple(c[1:]) == best[op][i] else 1.0 for i, c in enumerate(classes))

    monkeypatch.setattr(autotune, "_time", fake_time)
    vo = np.array([0, 1000, 20_000, 300_000], np.int64)
    path = str(tmp_path / "tuned.json")
    got = autotune.tune(300_000, {0: (None, None), 1: (None, None)}, vo,
                        {0: (None, np.zeros(4, np.int64)), 1: (None, np.zeros(4, np.int64))}, path=path)
    for op in (0, 1):
        assert [tuple(c[1:]) for c in got[op]] == [best[op][i] for i in range(3)]
        assert [c[0] for c in got[op]] == [c[0] for c in DEFAULT_CLASSES]
    sig = autotune.signature(vo)
    assert autotune.load(sig, path) == got
    assert autotune.load(autotune.signature(np.array([0, 5, 10], np.int64)), path) is None
