"""On-disk caches of generated graphs and of oracle results (CPU): a cached graph and a cached
result equal the freshly computed ones, the keys separate different recipes and arguments, and
calls without a key are never cached."""
import os

import numpy as np

import oracle
from paper_1911_09135_gb300 import graphgen as gg


def test_graph_cache_roundtrip(tmp_path, monkeypatch):
    fresh = gg.rmat(10, 16 << 10, 5, symmetrize=True, weighted=True, n_hubs=2, hub_degree=300)
    monkeypatch.setenv(gg.CACHE_ENV, str(tmp_path))
    a = gg.rmat(10, 16 << 10, 5, symmetrize=True, weighted=True, n_hubs=2, hub_degree=300)
    files = os.listdir(tmp_path)
    assert len(files) == 1 and files[0] == a.key + ".npz"
    b = gg.rmat(10, 16 << 10, 5, symmetrize=True, weighted=True, n_hubs=2, hub_degree=300)
    for g in (a, b):
        assert g.key == fresh.key and g.n == fresh.n and g.symmetric
        assert np.array_equal(g.offsets, fresh.offsets) and np.array_equal(g.indices, fresh.indices)
        assert np.array_equal(g.weights, fresh.weights) and np.array_equal(g.hubs, fresh.hubs)
    c = gg.rmat(10, 16 << 10, 6, symmetrize=True, weighted=True, n_hubs=2, hub_degree=300)
    assert c.key != a.key and len(os.listdir(tmp_path)) == 2


def test_oracle_cache_roundtrip(tmp_path, monkeypatch):
    g = gg.rmat(9, 16 << 9, 3, symmetrize=True, weighted=True)
    src = g.max_degree_vertex()
    want = (oracle.bfs(g.n, g.offsets, g.indices, src),
            oracle.sssp(g.n, g.offsets, g.indices, g.weights, src),
            oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000, assume_symmetric=True))
    monkeypatch.setenv(oracle.CACHE_ENV, str(tmp_path))
    assert oracle.bfs(g.n, g.offsets, g.indices, src) is not None and os.listdir(tmp_path) == []
    for _ in range(2):  # computed and stored, then read back
        got = (oracle.bfs(g.n, g.offsets, g.indices, src, cache_key=g.key),
               oracle.sssp(g.n, g.offsets, g.indices, g.weights, src, cache_key=g.key),
               oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000, assume_symmetric=True,
                               cache_key=g.key))
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert np.array_equal(got[2][0], want[2][0]) and got[2][1:] == want[2][1:]
        assert isinstance(got[2][1], int) and isinstance(got[2][2], float)
    assert len(os.listdir(tmp_path)) == 3
    other = oracle.bfs(g.n, g.offsets, g.indices, src + 7, cache_key=g.key)   # other arguments, own entry
    assert np.array_equal(other, oracle.bfs(g.n, g.offsets, g.indices, src + 7)) and len(os.listdir(tmp_path)) == 4
