"""Host logic of the server on CPU: the open-loop request generator and the latency statistics."""
import types

import numpy as np

from paper_1911_09135_gb300 import graphgen as gg
from paper_1911_09135_gb300 import serve


def _graphs():
    return [gg.rmat(sc, 16 << sc, 500 + i, symmetrize=True) for i, sc in enumerate((8, 9, 10))]


def test_poisson_requests_are_seeded_and_open_loop():
    gs = _graphs()
    a = serve.poisson_requests(gs, 20000, rate=2000.0, seed=5)
    b = serve.poisson_requests(gs, 20000, rate=2000.0, seed=5)
    assert [(r.arrival, r.graph, r.kind, r.src) for r in a] == [(r.arrival, r.graph, r.kind, r.src) for r in b]
    t = np.array([r.arrival for r in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000.0) < 0.03 / 2000.0        # exponential gaps, mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05          # coefficient of variation 1
    graphs = np.bincount([r.graph for r in a], minlength=3) / len(a)
    kinds = np.array([sum(r.kind == k for r in a) for k in serve.KINDS]) / len(a)
    assert np.all(np.abs(graphs - 1 / 3) < 0.02) and np.all(np.abs(kinds - 1 / 3) < 0.02)
    for r in a[:2000]:                                           # sources are non-isolated vertices
        assert gs[r.graph].degrees()[r.src] > 0
    c = serve.poisson_requests(gs, 200, rate=2000.0, seed=6)
    assert [r.src for r in c] != [r.src for r in a[:200]]


def test_latency_and_slot_statistics():
    reqs = [serve.Request(i, arrival=0.0, graph=i % 2, kind="bfs", src=0, done=(i + 1) * 1e-3)
            for i in range(100)]
    lat = serve.latency_stats(reqs)
    assert lat["p50_ms"] == np.percentile(np.arange(1, 101), 50)
    assert lat["p99_ms"] == np.percentile(np.arange(1, 101), 99)
    assert lat["max_ms"] == 100.0 and abs(lat["mean_ms"] - 50.5) < 1e-9
    g0 = types.SimpleNamespace(m=10, slots=[None], log=[(0.010, 32, 0, 1), (0.030, 4, 4, 0)])
    g1 = types.SimpleNamespace(m=20, slots=[None, None], log=[])
    st = serve.slot_stats(types.SimpleNamespace(graphs=[g0, g1]), reqs)
    assert st[0]["batches"] == 2 and st[0]["batch_ms_mean"] == 20.0 and st[0]["batch_size_mean"] == 20.5
    assert st[0]["requests"] == 50 and st[1]["slots"] == 2 and st[1]["batches"] == 0
