"""GPU parity at the full workload sizes, in the launch configuration bench.py times
(default parameters: hub threshold = threads of the LB kernel, cyclic distribution,
device-side round loop in a CUDA graph).

  rmat16 directed (scale 16, ef 16, seed 1):      bfs from 0 (and two more sources)
  rmat22 symmetrised (scale 22, ef 16, seed 2):   bfs + sssp from the max-degree vertex
  rmat24 + 16 hubs of 2^22 (seed 3), symmetrised: bfs, sssp, cc, pagerank, k-core (k = 32)

Integer results are compared element by element with the CPU oracle (sssp at scale
24 through the oracle's exact shortest-path certificate plus Dijkstra on a sample
check); PageRank must be within 1e-5 L1 of the FP64 oracle, and the error is printed.
With ALB_GRAPH_CACHE / ALB_ORACLE_CACHE set, the graphs and the oracle's results on them are
read from those directories when present (the cache keys name the generator's recipe).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1911_09135_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_09135_gb300 import alb  # noqa: E402

INF = 0xFFFFFFFF
NTHREADS = len(os.sched_getaffinity(0))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def make(g):
    return alb.Graph(g.n, dev(g.offsets), dev(g.indices),
                     dev(g.weights) if g.weights is not None else None, symmetric=g.symmetric)


def test_rmat16_directed_bfs():
    g = gg.rmat16_directed()
    with make(g) as G:
        o = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for src in (0, 1, 40000):
            G.bfs(src, o)
            assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, src))


@pytest.fixture(scope="module")
def rmat22():
    return gg.rmat22_sym()


def test_rmat22_bfs_sssp(rmat22):
    g = rmat22
    src = g.max_degree_vertex()
    with make(g) as G:
        o = torch.empty(g.n, dtype=torch.int32, device="cuda")
        G.bfs(src, o)
        assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, src, cache_key=g.key))
        G.sssp(src, o)
        assert np.array_equal(host(o), oracle.sssp(g.n, g.offsets, g.indices, g.weights, src,
                                                   cache_key=g.key))


@pytest.fixture(scope="module")
def rmat24():
    g = gg.rmat24_hubs_sym()
    G = make(g)
    yield g, G
    G.close()


def test_rmat24_bfs(rmat24):
    g, G = rmat24
    src = g.max_degree_vertex()
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o)
    got = host(o).copy()
    st = G.stats()
    assert st["hub_rounds"] > 0                 # the LB kernel ran at the default threshold
    assert np.array_equal(got, oracle.bfs(g.n, g.offsets, g.indices, src, cache_key=g.key))
    # threshold 0 (every active vertex huge) gives the identical result (Sec. 4.1)
    p = G.params()
    G.set_params(hub_threshold=0)
    G.bfs(src, o)
    assert np.array_equal(host(o), got)
    G.set_params(hub_threshold=p.hub_threshold)


def test_rmat24_sssp(rmat24):
    g, G = rmat24
    src = g.max_degree_vertex()
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.sssp(src, o)
    d = host(o).copy()
    assert oracle.check_sssp(g.n, g.offsets, g.indices, g.weights, src, d) == -1
    ref = oracle.sssp(g.n, g.offsets, g.indices, g.weights, src, cache_key=g.key)
    assert np.array_equal(d, ref)


def test_rmat24_cc(rmat24):
    g, G = rmat24
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.cc(o)
    assert np.array_equal(host(o), oracle.cc(g.n, g.offsets, g.indices, cache_key=g.key))


def test_rmat24_kcore(rmat24):
    g, G = rmat24
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.kcore(32, o)
    assert np.array_equal(host(o), oracle.kcore(g.n, g.offsets, g.indices, 32, cache_key=g.key))


def test_rmat24_pagerank(rmat24):
    """Within 1e-5 L1 of the FP64 oracle at the default threshold (the 16 hubs' in-edges in the
    LB kernel) and with no vertex huge (TWC only: one CTA sums a hub's 4.2M in-edges, a thread
    about 16K of them, which needs the compensated per-thread sums)."""
    g, G = rmat24
    r = torch.empty(g.n, dtype=torch.float32, device="cuda")
    ref, it_ref, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000,
                                     assume_symmetric=True, nthreads=NTHREADS, cache_key=g.key)
    p = G.params()
    for t in (p.hub_threshold, 1 << 40):
        G.set_params(hub_threshold=t)
        _, it, l1 = G.pagerank(0.85, 1e-6, 1000, r)
        x = r.cpu().numpy().astype(np.float64)
        err = float(np.abs(x - ref).sum())
        print(f"\npagerank rmat24 (threshold {t}): iterations gpu {it} oracle {it_ref}, "
              f"L1 |x_gpu - x_oracle| = {err:.3e}")
        assert err <= 1e-5
        assert abs(it - it_ref) <= 1 and l1 < 1e-6
        assert abs(x.sum() - 1.0) < 1e-4
    G.set_params(hub_threshold=p.hub_threshold)


def test_rmat22_batch_of_128_sources(rmat22):
    """128 uniform random sources (seed 4) in groups of 32 sharing CSR reads; every one of the
    256 results (bfs and sssp) is checked exactly by the oracle's certificates (a certificate
    accepts exactly the true levels / distances: the source at 0, no edge that could shorten a
    label, and every reached vertex with a tight in-edge), two of them also against the full
    oracle. The certificates run on a thread pool (the oracle's ctypes calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    g = rmat22
    rng = np.random.Generator(np.random.Philox(key=4))
    srcs = rng.integers(0, g.n, size=128).astype(np.uint32)
    with make(g) as G:
        out = torch.empty(128 * g.n, dtype=torch.int32, device="cuda")
        G.bfs_batch(srcs, out)
        lv = host(out).reshape(128, g.n).copy()
        G.sssp_batch(srcs, out)
        ds = host(out).reshape(128, g.n).copy()

    def certify(i):
        s = int(srcs[i])
        return (oracle.check_bfs(g.n, g.offsets, g.indices, s, lv[i]),
                oracle.check_sssp(g.n, g.offsets, g.indices, g.weights, s, ds[i]))

    with ThreadPoolExecutor(max_workers=NTHREADS) as ex:
        certs = list(ex.map(certify, range(128)))
    bad = [(i, v) for i, v in enumerate(certs) if v != (-1, -1)]
    assert not bad, bad[:8]
    for i in (0, 127):
        s = int(srcs[i])
        assert np.array_equal(lv[i], oracle.bfs(g.n, g.offsets, g.indices, s))
        assert np.array_equal(ds[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, s))


def test_512_small_graphs_in_one_traversal():
    parts = gg.small_graphs(512, seed=4)
    u, base = gg.disjoint_union(parts)
    srcs = base[:-1].astype(np.uint32)
    with make(u) as G:
        o = torch.empty(u.n, dtype=torch.int32, device="cuda")
        G.bfs_multi(srcs, o)
        lv = host(o).copy()
        G.sssp_multi(srcs, o)
        ds = host(o).copy()
    for i, p in enumerate(parts):
        sl = slice(int(base[i]), int(base[i + 1]))
        assert np.array_equal(lv[sl], oracle.bfs(p.n, p.offsets, p.indices, 0)), i
        if i % 8 == 0:
            assert np.array_equal(ds[sl], oracle.sssp(p.n, p.offsets, p.indices, p.weights, 0)), i
        else:
            assert oracle.check_sssp(p.n, p.offsets, p.indices, p.weights, 0, ds[sl]) == -1, i
