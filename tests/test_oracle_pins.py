"""Pins of the CPU oracle against things other than itself.

Each oracle function is checked against brute force on tiny graphs, a library
routine (scipy.sparse.csgraph / numpy.linalg) on medium ones, closed forms or
invariants, so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one test here.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from paper_1911_09135_gb300 import graphgen as gg
from tests import graphs

INF = oracle.INF


def dense_weights(g, unit=False):
    W = np.full((g.n, g.n), np.inf)
    np.fill_diagonal(W, 0.0)
    for u in range(g.n):
        for e in range(int(g.offsets[u]), int(g.offsets[u + 1])):
            v = int(g.indices[e])
            w = 1.0 if unit else float(g.weights[e])
            W[u, v] = min(W[u, v], w)
    return W


def floyd_warshall(W):
    D = W.copy()
    for k in range(D.shape[0]):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def to_u32_dist(row):
    return np.array([INF if np.isinf(x) else int(x) for x in row], dtype=np.uint32)


def scipy_matrix(g, weighted):
    data = g.weights.astype(np.float64) if weighted else np.ones(g.m)
    return sp.csr_matrix((data, g.indices.astype(np.int64), g.offsets.astype(np.int64)),
                         shape=(g.n, g.n))


SMALL = graphs.all_small() + [graphs.directed_cycle_tail()]


# ------------------------------------------------------------------ BFS

@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_bfs_vs_floyd_warshall(g):
    D = floyd_warshall(dense_weights(g, unit=True))
    for src in range(g.n):
        got = oracle.bfs(g.n, g.offsets, g.indices, src)
        assert np.array_equal(got, to_u32_dist(D[src])), (g.name, src)


@pytest.mark.parametrize("seed,directed", [(1, True), (2, False), (3, True)])
def test_bfs_vs_scipy(seed, directed):
    g = gg.random_graph(3000, 9000, seed, symmetrize=not directed, weighted=False)
    M = scipy_matrix(g, weighted=False)
    for src in (0, 17, 2999):
        ref = csg.shortest_path(M, directed=True, unweighted=True, indices=src)
        assert np.array_equal(oracle.bfs(g.n, g.offsets, g.indices, src), to_u32_dist(ref))


def test_bfs_rmat_vs_scipy():
    g = gg.rmat16_directed()
    ref = csg.shortest_path(scipy_matrix(g, False), directed=True, unweighted=True, indices=0)
    assert np.array_equal(oracle.bfs(g.n, g.offsets, g.indices, 0), to_u32_dist(ref))


def test_bfs_bad_source():
    g = graphs.path(4)
    with pytest.raises(oracle.OracleError):
        oracle.bfs(g.n, g.offsets, g.indices, 4)


# ----------------------------------------------------------------- SSSP

@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_sssp_vs_floyd_warshall(g):
    D = floyd_warshall(dense_weights(g))
    for src in range(g.n):
        got = oracle.sssp(g.n, g.offsets, g.indices, g.weights, src)
        assert np.array_equal(got, to_u32_dist(D[src])), (g.name, src)


@pytest.mark.parametrize("seed,directed", [(5, True), (6, False)])
def test_sssp_vs_scipy_dijkstra(seed, directed):
    g = gg.random_graph(4000, 16000, seed, symmetrize=not directed, weighted=True)
    M = scipy_matrix(g, weighted=True)
    for src in (0, 123, 3999):
        ref = csg.dijkstra(M, directed=True, indices=src)
        assert np.array_equal(oracle.sssp(g.n, g.offsets, g.indices, g.weights, src),
                              to_u32_dist(ref))


def test_sssp_rmat_vs_scipy():
    g = gg.rmat(14, 16 << 14, 11, symmetrize=True, weighted=True)
    src = g.max_degree_vertex()
    ref = csg.dijkstra(scipy_matrix(g, True), directed=True, indices=src)
    assert np.array_equal(oracle.sssp(g.n, g.offsets, g.indices, g.weights, src),
                          to_u32_dist(ref))


# ------------------------------------------------------------------- CC

def closure_labels(g):
    """Min id of each vertex's component, from the boolean reachability closure."""
    R = np.eye(g.n, dtype=bool)
    for u in range(g.n):
        for e in range(int(g.offsets[u]), int(g.offsets[u + 1])):
            R[u, int(g.indices[e])] = True
    R = R | R.T
    for _ in range(max(1, int(np.ceil(np.log2(max(g.n, 2)))) + 1)):
        R = R | ((R.astype(np.int64) @ R.astype(np.int64)) > 0)
    return np.array([int(np.nonzero(R[v])[0].min()) for v in range(g.n)], dtype=np.uint32)


@pytest.mark.parametrize("g", graphs.all_small(), ids=lambda g: g.name)
def test_cc_vs_closure(g):
    assert np.array_equal(oracle.cc(g.n, g.offsets, g.indices), closure_labels(g))


@pytest.mark.parametrize("seed", [7, 8])
def test_cc_vs_scipy(seed):
    g = gg.random_graph(20000, 15000, seed, symmetrize=True, weighted=False)
    _, lab = csg.connected_components(scipy_matrix(g, False), directed=False)
    # canonical label: smallest vertex id of the component
    mins = np.full(lab.max() + 1, np.iinfo(np.int64).max)
    np.minimum.at(mins, lab, np.arange(g.n))
    assert np.array_equal(oracle.cc(g.n, g.offsets, g.indices), mins[lab].astype(np.uint32))


# ------------------------------------------------------------- PageRank

def pagerank_dense_solve(g, d):
    """Fixed point of x = (1-d)/N + d (P^T x + (dangling . x)/N), by a dense linear solve."""
    n = g.n
    deg = g.degrees().astype(np.float64)
    A = np.zeros((n, n))
    for u in range(n):
        for e in range(int(g.offsets[u]), int(g.offsets[u + 1])):
            A[int(g.indices[e]), u] += 1.0 / deg[u]
    dangling = (deg == 0).astype(np.float64)
    G = A + np.outer(np.ones(n), dangling) / n
    return np.linalg.solve(np.eye(n) - d * G, np.full(n, (1.0 - d) / n))


@pytest.mark.parametrize("seed,sym,m", [(1, False, 400), (2, True, 110), (3, False, 300)])
def test_pagerank_vs_dense_solve(seed, sym, m):
    g = gg.random_graph(150, m, seed, symmetrize=sym, weighted=False)
    assert (g.degrees() == 0).any()  # dangling vertices present
    x, it, l1 = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-14, 10000,
                                assume_symmetric=sym)
    ref = pagerank_dense_solve(g, 0.85)
    assert np.abs(x - ref).sum() < 1e-11
    assert abs(x.sum() - 1.0) < 1e-12
    assert l1 < 1e-14


def test_pagerank_symmetric_shortcut_equals_transpose():
    g = gg.random_graph(500, 3000, 4, symmetrize=True, weighted=False)
    a = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-10, 1000, assume_symmetric=True)
    b = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-10, 1000, assume_symmetric=False)
    assert a[1] == b[1] and np.abs(a[0] - b[0]).max() < 1e-15


@pytest.mark.parametrize("g", [graphs.cycle(11), graphs.complete(7)], ids=lambda g: g.name)
def test_pagerank_regular_graph_is_uniform(g):
    x, it, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-12, 100)
    assert np.allclose(x, 1.0 / g.n, atol=1e-15, rtol=0)
    assert it == 1  # uniform start is already the fixed point


def test_pagerank_star_closed_form():
    N, d = 9, 0.85
    g = graphs.star(N)
    x, _, _ = oracle.pagerank(g.n, g.offsets, g.indices, d, 1e-15, 10000)
    # centre c, leaves l:  l = (1-d)/N + d c/(N-1),  c = (1-d)/N + d (N-1) l
    A = np.array([[1.0, -d / (N - 1)], [-d * (N - 1), 1.0]])
    l, c = np.linalg.solve(A, np.full(2, (1 - d) / N))
    assert abs(x[0] - c) < 1e-14 and np.allclose(x[1:], l, atol=1e-14, rtol=0)


def test_pagerank_isolated_vertices_count_in_n():
    g = gg.from_edges(4, [(0, 1)], symmetrize=True)  # vertices 2, 3 isolated (dangling)
    x, _, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-15, 10000)
    ref = pagerank_dense_solve(g, 0.85)
    assert np.abs(x - ref).sum() < 1e-13 and abs(x.sum() - 1) < 1e-13


def test_pagerank_stopping_rule():
    g = gg.random_graph(300, 1500, 9, symmetrize=True, weighted=False)
    _, it6, l16 = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000)
    _, it5, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, it6 - 1)
    assert l16 < 1e-6 and it5 == it6 - 1
    _, _, l1prev = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 0.0, it6 - 1)
    assert l1prev >= 1e-6  # the iteration before the stop had not converged


# --------------------------------------------------------------- k-core

def kcore_brute(g, k):
    """Union of all vertex subsets whose induced minimum degree is >= k (n <= 14)."""
    n = g.n
    adj = [set(int(x) for x in g.indices[g.offsets[u]:g.offsets[u + 1]]) for u in range(n)]
    best = np.zeros(n, dtype=np.uint32)
    for mask in range(1, 1 << n):
        S = [v for v in range(n) if mask >> v & 1]
        Sset = set(S)
        if all(len(adj[v] & Sset) >= k for v in S):
            best[S] = 1
    return best


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_kcore_vs_subset_enumeration(seed, k):
    g = gg.random_graph(12, 26, seed, symmetrize=True, weighted=False)
    assert np.array_equal(oracle.kcore(g.n, g.offsets, g.indices, k), kcore_brute(g, k))


@pytest.mark.parametrize("g", graphs.all_small(), ids=lambda g: g.name)
def test_kcore_small_graphs(g):
    for k in (0, 1, 2, 3, 6):
        assert np.array_equal(oracle.kcore(g.n, g.offsets, g.indices, k), kcore_brute(g, k))


def test_kcore_vs_networkx():
    nx = pytest.importorskip("networkx")
    g = gg.rmat(12, 16 << 12, 21, symmetrize=True)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), g.degrees().astype(np.int64))
    G.add_edges_from(zip(src.tolist(), g.indices.tolist()))
    core = nx.core_number(G)  # Batagelj-Zaversnik core numbers
    for k in (1, 8, 32, 64):
        ref = np.array([1 if core[v] >= k else 0 for v in range(g.n)], dtype=np.uint32)
        assert np.array_equal(oracle.kcore(g.n, g.offsets, g.indices, k), ref)


# --------------------------------------------------------- Algorithm 1

def test_inspect_definition_random():
    g = gg.rmat(12, 16 << 12, 5, symmetrize=True)
    rng = np.random.default_rng(0)
    wl = rng.permutation(g.n)[:1500].astype(np.uint32)
    deg = g.degrees().astype(np.int64)
    for t in (0, 1, 31, 32, 33, 255, 256, 257, 1000, int(deg.max()), int(deg.max()) + 1):
        work, prefix, b, counts = oracle.inspect(g.n, g.offsets, wl, t, 32, 256)
        dw = deg[wl]
        huge = dw >= t
        assert np.array_equal(work, wl[huge])                       # worklist order kept
        assert np.array_equal(prefix, np.concatenate([[0], np.cumsum(dw[huge])]).astype(np.uint64))
        exp = np.where(huge, 3, np.where(dw < 32, 0, np.where(dw < 256, 1, 2)))
        assert np.array_equal(b, exp.astype(np.uint8))
        assert counts.tolist() == [int((exp == c).sum()) for c in range(4)]
    # threshold 0: every active vertex is huge; threshold > max degree: none is (Sec. 4.1)
    assert oracle.inspect(g.n, g.offsets, wl, 0)[3][3] == len(wl)
    assert oracle.inspect(g.n, g.offsets, wl, int(deg.max()) + 1)[3][3] == 0


# --------------------------------------------------------- Algorithm 2

def _hub_setup(threshold, seed=3):
    g = gg.rmat(11, 16 << 11, seed, symmetrize=True)
    wl = np.arange(g.n, dtype=np.uint32)
    work, prefix, _, _ = oracle.inspect(g.n, g.offsets, wl, threshold)
    return g, work, prefix


@pytest.mark.parametrize("policy", ["cyclic", "blocked"])
@pytest.mark.parametrize("threshold,p", [(0, 64), (20, 96), (64, 64), (200, 1000)])
def test_lb_edges_cover_each_huge_edge_once(policy, threshold, p):
    g, work, prefix = _hub_setup(threshold)
    e = int(prefix[-1])
    seen_k, pairs = [], []
    for i in range(p):
        ks, ss, ds = oracle.lb_edges(g.offsets, g.indices, work, prefix, p, i, policy)
        if policy == "cyclic":
            assert np.all(ks % p == i)
        else:
            c = -(-e // p)
            assert np.array_equal(ks, np.arange(i * c, min(e, (i + 1) * c), dtype=np.uint64))
        seen_k.append(ks)
        pairs.append(np.stack([ss, ds], axis=1).astype(np.int64))
    ks = np.sort(np.concatenate(seen_k))
    assert np.array_equal(ks, np.arange(e, dtype=np.uint64))
    got = np.concatenate(pairs)
    exp = np.concatenate([
        np.stack([np.full(int(g.offsets[u + 1] - g.offsets[u]), u),
                  g.indices[g.offsets[u]:g.offsets[u + 1]]], axis=1) for u in work]).astype(np.int64)
    key = lambda a: a[np.lexsort((a[:, 1], a[:, 0]))]
    assert np.array_equal(key(got), key(exp))


def test_cyclic_at_most_two_sources_per_warp_when_threshold_ge_threads():
    # Sec. 4.1 "Threshold": with threshold = number of threads, the 32 consecutive edges a
    # warp takes in one cyclic sweep belong to at most two huge vertices.
    p = 256
    g, work, prefix = _hub_setup(p)
    assert len(work) >= 2
    e = int(prefix[-1])
    src_of_k = np.empty(e, dtype=np.int64)
    for i in range(p):
        ks, ss, _ = oracle.lb_edges(g.offsets, g.indices, work, prefix, p, i, "cyclic")
        src_of_k[ks.astype(np.int64)] = ss
    for base in range(0, e, 32):
        assert len(np.unique(src_of_k[base:base + 32])) <= 2
    # below the rule the bound no longer holds
    g2, work2, prefix2 = _hub_setup(2)
    e2 = int(prefix2[-1])
    src2 = np.repeat(work2, np.diff(prefix2.astype(np.int64)))
    assert max(len(np.unique(src2[b:b + 32])) for b in range(0, e2, 32)) > 2


# ---------------------------------------------------- certificates

@pytest.mark.parametrize("seed", [1, 2])
def test_check_bfs_accepts_truth_and_rejects_planted_errors(seed):
    g = gg.rmat(12, 16 << 12, seed, symmetrize=(seed == 2))
    src = g.max_degree_vertex()
    lv = oracle.bfs(g.n, g.offsets, g.indices, src)
    assert oracle.check_bfs(g.n, g.offsets, g.indices, src, lv) == -1
    reached = np.nonzero((lv != INF) & (lv > 0))[0]
    unreached = np.nonzero(lv == INF)[0]
    rng = np.random.default_rng(seed)
    for _ in range(20):
        bad = lv.copy()
        v = int(rng.choice(reached))
        delta = int(rng.choice([1, -1])) if bad[v] > 1 else 1
        bad[v] = np.uint32(int(bad[v]) + delta)
        assert oracle.check_bfs(g.n, g.offsets, g.indices, src, bad) != -1
    if unreached.size:
        bad = lv.copy(); bad[unreached[0]] = 5
        assert oracle.check_bfs(g.n, g.offsets, g.indices, src, bad) != -1
    bad = lv.copy(); bad[reached[0]] = INF
    assert oracle.check_bfs(g.n, g.offsets, g.indices, src, bad) != -1
    bad = lv.copy(); bad[src] = 1
    assert oracle.check_bfs(g.n, g.offsets, g.indices, src, bad) != -1


def test_check_sssp_accepts_truth_and_rejects_planted_errors():
    g = gg.rmat(12, 16 << 12, 4, symmetrize=True, weighted=True)
    src = g.max_degree_vertex()
    d = oracle.sssp(g.n, g.offsets, g.indices, g.weights, src)
    assert oracle.check_sssp(g.n, g.offsets, g.indices, g.weights, src, d) == -1
    reached = np.nonzero((d != INF) & (d > 0))[0]
    rng = np.random.default_rng(3)
    for delta in (1, -1, 2, -2, 7):
        for _ in range(10):
            bad = d.copy()
            v = int(rng.choice(reached))
            bad[v] = max(1, int(bad[v]) + delta)
            if bad[v] == d[v]:
                continue
            assert oracle.check_sssp(g.n, g.offsets, g.indices, g.weights, src, bad) != -1
    bad = d.copy(); bad[reached[0]] = INF
    assert oracle.check_sssp(g.n, g.offsets, g.indices, g.weights, src, bad) != -1


# ------------------------------------------------- paper worked example

def test_fig2_worked_example():
    """Golden values stated in Sec. 4.1 (Search, Fig. 2): v0 owns the first 40 huge edges and
    thread T4 processes edge e4 under the cyclic distribution, whose source is v0; threads
    T0..T19 take the consecutive edges E0..E19."""
    import json, os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig2_cyclic.json")))
    degs = fx["huge_degrees"]
    n = len(degs) + max(degs)
    edges = []
    for v, dv in enumerate(degs):
        edges += [(v, len(degs) + j) for j in range(dv)]
    g = gg.from_edges(n, edges, symmetrize=False)
    wl = np.arange(len(degs), dtype=np.uint32)
    work, prefix, _, _ = oracle.inspect(g.n, g.offsets, wl, fx["threshold"])
    assert prefix.tolist()[:2] == [0, fx["v0_edges"]]
    p = fx["threads"]
    ks, ss, _ = oracle.lb_edges(g.offsets, g.indices, work, prefix, p, fx["thread"], "cyclic")
    assert int(ks[0]) == fx["edge"] and int(ss[0]) == fx["source"]
    firsts = [int(oracle.lb_edges(g.offsets, g.indices, work, prefix, p, i, "cyclic")[0][0])
              for i in range(20)]
    assert firsts == list(range(20))
