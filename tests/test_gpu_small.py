"""GPU parity on small graphs: every app through the C ABI against the CPU oracle.

Integer apps must match bit for bit; PageRank within 1e-5 L1 of the FP64 oracle.
Thresholds and TWC cut-offs are forced so that tiny graphs reach every bin and
the LB kernel, in both the CUDA-graph and the host-loop execution modes.
"""
import numpy as np
import pytest

import oracle
from paper_1911_09135_gb300 import graphgen as gg
from tests import graphs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_09135_gb300 import alb  # noqa: E402

PR_TOL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def make(g):
    return alb.Graph(g.n, dev(g.offsets), dev(g.indices),
                     dev(g.weights) if g.weights is not None else None, symmetric=g.symmetric)


def run_all(G, g, src, k=3):
    out = {}
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o); out["bfs"] = host(o).copy()
    if g.weights is not None:
        G.sssp(src, o); out["sssp"] = host(o).copy()
    if g.symmetric:
        G.cc(o); out["cc"] = host(o).copy()
        G.kcore(k, o); out["kcore"] = host(o).copy()
    G.sync()
    return out


def oracle_all(g, src, k=3):
    out = {"bfs": oracle.bfs(g.n, g.offsets, g.indices, src)}
    if g.weights is not None:
        out["sssp"] = oracle.sssp(g.n, g.offsets, g.indices, g.weights, src)
    if g.symmetric:
        out["cc"] = oracle.cc(g.n, g.offsets, g.indices)
        out["kcore"] = oracle.kcore(g.n, g.offsets, g.indices, k)
    return out


SETTINGS = [
    dict(hub_threshold=-1),
    dict(hub_threshold=3, twc_warp_min=1, twc_cta_min=2, block_size=128),
    dict(hub_threshold=5, twc_warp_min=2, twc_cta_min=3, block_size=512, distribution=1),
    dict(hub_threshold=0),
    dict(hub_threshold=1),
    dict(hub_threshold=3, twc_warp_min=1, twc_cta_min=2),
    dict(hub_threshold=8, twc_warp_min=2, twc_cta_min=4, distribution=1),
    dict(hub_threshold=2, exec_mode=1),
    dict(hub_threshold=1 << 40),
    dict(hub_threshold=4, grid_blocks=3),
]


@pytest.mark.parametrize("g", graphs.all_small() + [graphs.directed_cycle_tail()],
                         ids=lambda g: g.name)
@pytest.mark.parametrize("setting", SETTINGS, ids=lambda s: ",".join(f"{k}={v}" for k, v in s.items()))
def test_small_graphs_all_apps(g, setting):
    G = make(g)
    G.set_params(**setting)
    for src in sorted({0, g.n - 1, g.n // 2}):
        got = run_all(G, g, src)
        ref = oracle_all(g, src)
        for app in ref:
            assert np.array_equal(got[app], ref[app]), (app, src)
    G.close()


@pytest.fixture(scope="module")
def rmat13():
    return gg.rmat(13, 16 << 13, 21, symmetrize=True, weighted=True, n_hubs=4, hub_degree=3000)


@pytest.mark.parametrize("t", [0, 1, 31, 32, 33, 255, 256, 257, 2999, 3000, 3001, -1, 1 << 33])
def test_threshold_sweep_identical_results(rmat13, t):
    """Sec. 4.1: t = 0 (all huge) .. t > max degree (plain TWC) must give identical output."""
    g = rmat13
    src = g.max_degree_vertex()
    G = make(g)
    G.set_params(hub_threshold=t)
    got = run_all(G, g, src, k=16)
    ref = oracle_all(g, src, k=16)
    for app in ref:
        assert np.array_equal(got[app], ref[app]), app
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o)
    st = G.stats()
    # the source is the max-degree vertex: it is huge whenever t <= max degree
    assert (st["hub_rounds"] > 0) == (0 <= t <= int(g.degrees().max()))
    assert st["edges_twc"] + st["edges_lb"] == int(g.degrees()[host(o) != 0xFFFFFFFF].sum())
    G.close()


@pytest.mark.parametrize("block_size", [128, 256, 512])
@pytest.mark.parametrize("t", [-1, 0, 64, 3000])
def test_cta_sizes_identical_results(rmat13, block_size, t):
    """The round kernels built for 128, 256 and 512 threads per CTA give the oracle's results at
    every threshold; the paper's rule follows the LB kernel's thread count."""
    g = rmat13
    src = g.max_degree_vertex()
    G = make(g)
    G.set_params(hub_threshold=t, block_size=block_size)
    got = run_all(G, g, src, k=16)
    ref = oracle_all(g, src, k=16)
    for app in ref:
        assert np.array_equal(got[app], ref[app]), app
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o)
    st = G.stats()
    assert st["block_size"] == block_size and st["lb_threads"] % block_size == 0
    if t == -1:
        assert st["hub_threshold"] == st["lb_threads"]
    srcs = np.array([0, 7, 100, 4095, src], dtype=np.uint32)   # the batched path takes it too
    out = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    G.sssp_batch(srcs, out)
    res = host(out).reshape(len(srcs), g.n)
    for i, s in enumerate(srcs):
        assert np.array_equal(res[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, int(s))), i
    G.close()


def test_cta_size_argument_errors(rmat13):
    G = make(rmat13)
    for bad in (64, 100, 1024):
        with pytest.raises(alb.AlbError) as e:
            G.set_params(block_size=bad)
        assert e.value.code == 1
    G.close()


@pytest.mark.parametrize("distribution", [0, 1])
@pytest.mark.parametrize("exec_mode", [0, 1])
def test_rmat_directed_bfs_and_modes(distribution, exec_mode):
    g = gg.rmat16_directed()
    G = make(g)
    G.set_params(hub_threshold=2048, distribution=distribution, exec_mode=exec_mode)
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for src in (0, 1, 12345):
        G.bfs(src, o)
        assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, src))
    G.close()


@pytest.mark.parametrize("t", [-1, 0, 64, 1 << 33])
@pytest.mark.parametrize("exec_mode", [0, 1])
def test_pagerank_small(rmat13, t, exec_mode):
    g = rmat13
    G = make(g)
    G.set_params(hub_threshold=t, exec_mode=exec_mode)
    r = torch.empty(g.n, dtype=torch.float32, device="cuda")
    _, it, l1 = G.pagerank(0.85, 1e-6, 1000, r)
    ref, it_ref, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000,
                                     assume_symmetric=True)
    err = float(np.abs(r.cpu().numpy().astype(np.float64) - ref).sum())
    assert err <= PR_TOL, err
    assert abs(it - it_ref) <= 1 and l1 < 1e-6
    G.close()


def test_pagerank_deterministic_and_threshold_independent_within_tol(rmat13):
    g = rmat13
    G = make(g)
    r1 = torch.empty(g.n, dtype=torch.float32, device="cuda")
    r2 = torch.empty(g.n, dtype=torch.float32, device="cuda")
    G.set_params(hub_threshold=64)
    G.pagerank(0.85, 1e-6, 1000, r1)
    G.pagerank(0.85, 1e-6, 1000, r2)
    assert torch.equal(r1, r2)  # fixed reduction order: bit-reproducible
    G.close()


def test_pagerank_edge_cases():
    for g in graphs.all_small():
        G = make(g)
        G.set_params(hub_threshold=2)
        r = torch.empty(g.n, dtype=torch.float32, device="cuda")
        G.pagerank(0.85, 1e-8, 500, r)
        ref, _, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-8, 500, assume_symmetric=True)
        assert float(np.abs(r.cpu().numpy() - ref).sum()) <= PR_TOL, g.name
        # max_iter = 0 returns the starting vector
        G.pagerank(0.85, 1e-8, 0, r)
        assert np.allclose(r.cpu().numpy(), 1.0 / g.n)
        G.close()


def test_host_buffers_through_the_abi(rmat13):
    g = rmat13
    G = alb.Graph(g.n, g.offsets, g.indices, g.weights, symmetric=True)  # host CSR input
    src = 5
    lv = G.bfs(src)  # host output
    assert np.array_equal(lv, oracle.bfs(g.n, g.offsets, g.indices, src))
    d = G.sssp(src)
    assert np.array_equal(d, oracle.sssp(g.n, g.offsets, g.indices, g.weights, src))
    x, it, l1 = G.pagerank()
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000, assume_symmetric=True)
    assert np.abs(x - ref).sum() <= PR_TOL
    G.close()


def test_inspect_matches_algorithm_1(rmat13):
    g = rmat13
    G = make(g)
    rng = np.random.default_rng(1)
    wl = rng.permutation(g.n)[:5000].astype(np.uint32)
    for t in (0, 1, 32, 100, 1000, 1 << 33):
        G.set_params(hub_threshold=t)
        work, prefix, bins, counts = G.inspect(wl)
        ow, op, ob, oc = oracle.inspect(g.n, g.offsets, wl, min(t, 0xFFFFFFFF))
        assert np.array_equal(bins, ob) and np.array_equal(counts, oc)
        # the huge set is unique; its order is the device's append order
        assert np.array_equal(np.sort(work), np.sort(ow))
        deg = g.degrees().astype(np.uint64)
        assert np.array_equal(prefix.astype(np.uint64),
                              np.concatenate([[0], np.cumsum(deg[work])]).astype(np.uint64))
    G.close()


@pytest.mark.parametrize("distribution", [0, 1])
@pytest.mark.parametrize("grid", [0, 5])
def test_lb_kernel_assignment_is_algorithm_2(rmat13, distribution, grid):
    """The LB kernel itself deals position k to the thread Algorithm 2 names."""
    g = rmat13
    G = make(g)
    G.set_params(hub_threshold=200, distribution=distribution, grid_blocks=grid)
    p = G.stats()["lb_threads"]
    wl = np.arange(g.n, dtype=np.uint32)
    work, prefix, _, _ = oracle.inspect(g.n, g.offsets, wl, 200)
    src, dst, thr = G.lb_trace(work, prefix.astype(np.uint32))
    e = int(prefix[-1])
    policy = "cyclic" if distribution == 0 else "blocked"
    exp_src = np.empty(e, dtype=np.uint32)
    exp_dst = np.empty(e, dtype=np.uint32)
    exp_thr = np.empty(e, dtype=np.uint32)
    busy = min(p, e) if policy == "cyclic" else -(-e // -(-e // p))  # threads holding positions
    for i in range(busy):
        ks, ss, ds = oracle.lb_edges(g.offsets, g.indices, work, prefix, p, i, policy)
        exp_src[ks.astype(np.int64)] = ss
        exp_dst[ks.astype(np.int64)] = ds
        exp_thr[ks.astype(np.int64)] = i
    assert np.array_equal(src, exp_src)
    assert np.array_equal(dst, exp_dst)
    assert np.array_equal(thr, exp_thr)
    G.close()


def test_lb_trace_rejects_inconsistent_prefix(rmat13):
    g = rmat13
    G = make(g)
    work = np.array([0, 1], dtype=np.uint32)
    bad = np.array([0, 5, 10], dtype=np.uint32)
    with pytest.raises(alb.AlbError):
        G.lb_trace(work, bad)
    G.close()


def test_argument_and_capability_errors():
    g = graphs.directed_cycle_tail()
    G = make(g)
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(alb.AlbError) as e:
        G.bfs(g.n, o)
    assert e.value.code == 1
    with pytest.raises(alb.AlbError) as e:
        G.cc(o)
    assert e.value.code == 6
    with pytest.raises(alb.AlbError) as e:
        G.kcore(2, o)
    assert e.value.code == 6
    G.close()
    g2 = gg.from_edges(3, [(0, 1), (1, 2)], symmetrize=True)
    G2 = make(g2)
    with pytest.raises(alb.AlbError) as e:
        G2.sssp(0, o)
    assert e.value.code == 7
    G2.close()
    # an index >= n in the CSR is caught at creation
    off = np.array([0, 1, 2], dtype=np.uint32)
    idx = np.array([1, 7], dtype=np.uint32)
    with pytest.raises(alb.AlbError) as e:
        alb.Graph(2, off, idx)
    assert e.value.code == 8
    # offsets[n] != m
    with pytest.raises(alb.AlbError) as e:
        alb.alb_graph_create(2, 1, off, idx[:1])
    assert e.value.code == 1


def test_round_limit_reports_timeout():
    g = graphs.path(9)
    G = make(g)
    G.set_params(max_rounds=3)
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(0, o)
    with pytest.raises(alb.AlbError) as e:
        G.sync()
    assert e.value.code == 4
    G.set_params(max_rounds=0)
    G.bfs(0, o)
    G.sync()
    assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, 0))
    G.close()


def test_batch_matches_single_source(rmat13):
    g = rmat13
    G = make(g)
    srcs = np.array([0, 7, 100, 4095], dtype=np.uint32)
    out = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    G.bfs_batch(torch.from_numpy(srcs.view(np.int32)).cuda(), out)
    res = host(out).reshape(len(srcs), g.n)
    for i, s in enumerate(srcs):
        assert np.array_equal(res[i], oracle.bfs(g.n, g.offsets, g.indices, int(s)))
    G.sssp_batch(srcs, out)
    res = host(out).reshape(len(srcs), g.n)
    for i, s in enumerate(srcs):
        assert np.array_equal(res[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, int(s)))
    G.close()


@pytest.mark.parametrize("exec_mode", [0, 1])
@pytest.mark.parametrize("t", [-1, 0, 64, 1 << 33])
def test_batch_groups_ragged_and_duplicates(rmat13, t, exec_mode):
    """40 sources = a full group of 32 and a ragged group of 8, with repeated sources; in the
    CUDA-graph mode and the host loop (one launch per kernel)."""
    g = rmat13
    G = make(g)
    G.set_params(hub_threshold=t, exec_mode=exec_mode, profile=exec_mode)
    rng = np.random.default_rng(7)
    srcs = rng.integers(0, g.n, size=40).astype(np.uint32)
    srcs[5] = srcs[3]
    srcs[33] = srcs[3]
    out = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    G.bfs_batch(srcs, out)
    res = host(out).reshape(len(srcs), g.n).copy()
    G.sssp_batch(srcs, out)
    res2 = host(out).reshape(len(srcs), g.n).copy()
    if exec_mode == 1:
        st = G.stats()   # the host loop times every round kernel of both groups
        assert st["n_inspect"] > st["rounds"] > 0 and st["ms_inspect"] > 0   # rounds: the last group's
    for i, s in enumerate(srcs):
        assert np.array_equal(res[i], oracle.bfs(g.n, g.offsets, g.indices, int(s))), i
        assert np.array_equal(res2[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, int(s))), i
    G.close()


def test_batch_host_output_and_directed():
    g = gg.rmat16_directed()
    G = alb.Graph(g.n, g.offsets, g.indices)
    srcs = [0, 1, 2, 40000, 65535]
    res = G.bfs_batch(srcs).reshape(len(srcs), g.n)
    for i, s in enumerate(srcs):
        assert np.array_equal(res[i], oracle.bfs(g.n, g.offsets, g.indices, s))
    G.close()


def test_multi_source_is_min_over_sources(rmat13):
    g = rmat13
    G = make(g)
    srcs = np.array([0, 100, 5000, 100], dtype=np.uint32)
    lv = G.bfs_multi(srcs)
    d = G.sssp_multi(srcs)
    exp_l = np.minimum.reduce([oracle.bfs(g.n, g.offsets, g.indices, int(s)) for s in srcs])
    exp_d = np.minimum.reduce([oracle.sssp(g.n, g.offsets, g.indices, g.weights, int(s)) for s in srcs])
    assert np.array_equal(lv, exp_l) and np.array_equal(d, exp_d)
    G.close()


@pytest.mark.parametrize("t,exec_mode", [(-1, 0), (0, 0), (1 << 33, 0), (-1, 1)])
def test_disjoint_union_of_many_graphs(t, exec_mode):
    rng = np.random.default_rng(3)
    parts = [gg.rmat(int(sc), int(16 << sc), 100 + i, symmetrize=True, weighted=True)
             for i, sc in enumerate(rng.integers(4, 11, size=25))]
    parts += [graphs.star(40), graphs.path(30), graphs.empty(3)]
    u, base = gg.disjoint_union(parts)
    G = make(u)
    G.set_params(hub_threshold=t, exec_mode=exec_mode)
    srcs = base[:-1].astype(np.uint32)  # vertex 0 of every graph
    lv = G.bfs_multi(srcs)
    d = G.sssp_multi(srcs)
    for i, p in enumerate(parts):
        sl = slice(int(base[i]), int(base[i + 1]))
        assert np.array_equal(lv[sl], oracle.bfs(p.n, p.offsets, p.indices, 0)), i
        assert np.array_equal(d[sl], oracle.sssp(p.n, p.offsets, p.indices, p.weights, 0)), i
    G.close()


def test_batch_argument_errors(rmat13):
    g = rmat13
    G = make(g)
    with pytest.raises(alb.AlbError) as e:
        G.bfs_batch(np.array([0, g.n], dtype=np.uint32))
    assert e.value.code == 1
    with pytest.raises(alb.AlbError):
        G.bfs_multi(np.array([g.n + 5], dtype=np.uint32))
    # device-memory sources are checked on the device: the bad one is skipped, the error latched
    bad = torch.tensor([0, g.n + 5], dtype=torch.int32, device="cuda")
    out = torch.empty(2 * g.n, dtype=torch.int32, device="cuda")
    G.bfs_batch(bad, out)
    with pytest.raises(alb.AlbError) as e:
        G.sync()
    assert e.value.code == 1
    assert np.array_equal(host(out)[:g.n], oracle.bfs(g.n, g.offsets, g.indices, 0))
    G.close()


@pytest.mark.parametrize("app", ["bfs", "sssp", "cc", "pr", "kcore"])
def test_autotune_keeps_results_exact(rmat13, app):
    g = rmat13
    G = make(g)
    src = g.max_degree_vertex()
    p, ms = G.autotune(app, src, reps=2)
    assert ms > 0
    assert p.hub_threshold in [-1, 1 << 40] + [1 << k for k in range(8, 21, 2)]
    assert p.twc_cta_min in (128, 256, 512, 1024) and p.twc_warp_min in (16, 32, 64)
    assert p.block_size in (128, 256, 512)
    q = G.params(app)
    assert (q.hub_threshold, q.twc_cta_min, q.twc_warp_min, q.block_size) == \
        (p.hub_threshold, p.twc_cta_min, p.twc_warp_min, p.block_size)
    got = run_all(G, g, src, k=32)
    ref = oracle_all(g, src, k=32)
    for a in ref:
        assert np.array_equal(got[a], ref[a]), a
    G.close()


def test_per_app_params_are_independent(rmat13):
    g = rmat13
    G = make(g)
    G.set_app_params("sssp", hub_threshold=0, distribution=1)
    G.set_app_params("bfs", hub_threshold=1 << 40)
    assert G.params("sssp").hub_threshold == 0 and G.params("cc").hub_threshold == -1
    src = g.max_degree_vertex()
    got = run_all(G, g, src, k=8)
    ref = oracle_all(g, src, k=8)
    for a in ref:
        assert np.array_equal(got[a], ref[a]), a
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o)
    assert G.stats()["hub_rounds"] == 0          # bfs: never huge
    G.sssp(src, o)
    assert G.stats()["hub_threshold"] == 0       # sssp: every vertex huge
    G.close()


def test_clone_shares_the_csr_and_outlives_the_original(rmat13):
    g = rmat13
    G = make(g)
    G.set_app_params("bfs", hub_threshold=64)
    C = G.clone()
    assert C.params("bfs").hub_threshold == 64
    src = g.max_degree_vertex()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    o1 = torch.empty(g.n, dtype=torch.int32, device="cuda")
    o2 = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o1, stream=s1)          # the two handles run on different streams
    C.sssp(src, o2, stream=s2)
    torch.cuda.synchronize()
    assert np.array_equal(host(o1), oracle.bfs(g.n, g.offsets, g.indices, src))
    assert np.array_equal(host(o2), oracle.sssp(g.n, g.offsets, g.indices, g.weights, src))
    G.close()                          # the clone keeps the CSR alive
    C.cc(o1)
    C.sync()
    assert np.array_equal(host(o1), oracle.cc(g.n, g.offsets, g.indices))
    C.close()


def pull_cut_edges(g, t, wmin, cmin, nblocks, item_cost=3):
    """Edges per CTA of the PageRank pull under its static cut: every bin (CTA, warp, thread; each
    in vertex order) is cut separately, item cost degree + item_cost, and CTA b takes the bin's
    items whose inclusive cost prefix lies in (T_b, T_{b+1}], T_b = P0 + floor(C * b / G)."""
    deg = np.diff(g.offsets.astype(np.int64))
    hub = deg >= t
    cta = ~hub & (deg >= cmin)
    warp = ~hub & ~cta & (deg >= wmin)
    thr = ~hub & ~cta & ~warp
    out = np.zeros(nblocks, dtype=np.uint64)
    b = np.arange(nblocks + 1, dtype=np.int64)
    for sel in (cta, warp, thr):
        d = deg[np.flatnonzero(sel)]
        if d.size == 0:
            continue
        incl = np.cumsum(d + item_cost)
        C = int(incl[-1])
        T = (C // nblocks) * b + ((C % nblocks) * b) // nblocks
        cut = np.searchsorted(incl, T, side="right")
        e = np.concatenate([[0], np.cumsum(d)])
        out += (e[cut[1:]] - e[cut[:-1]]).astype(np.uint64)
    return out


def test_cta_loads_account_for_every_edge(rmat13):
    """Per-CTA counters (the paper's thread-block load measure) sum to the edges expanded."""
    g = rmat13
    G = make(g)
    src = g.max_degree_vertex()
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.set_params(hub_threshold=512, cta_stats=1)
    G.bfs(src, o)
    st = G.stats()
    twc, lb = G.cta_loads()
    assert len(twc) == st["grid_blocks"] and len(lb) == st["lb_threads"] // st["block_size"]
    assert int(twc.sum()) == st["edges_twc"] and int(lb.sum()) == st["edges_lb"] > 0
    assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, src))
    # the cyclic LB kernel spreads huge-vertex edges evenly: CTA loads differ by <= 256 * rounds
    assert int(lb.max()) - int(lb.min()) <= 256 * st["hub_rounds"]
    r = torch.empty(g.n, dtype=torch.float32, device="cuda")
    _, it, _ = G.pagerank(0.85, 1e-6, 1000, r)
    twc, lb = G.cta_loads()
    assert int(twc.sum()) + int(lb.sum()) == g.m * it
    # the pull kernel's CTAs take the cost-balanced contiguous ranges, counted per iteration
    p = G.params()
    exp = pull_cut_edges(g, 512, p.twc_warp_min, p.twc_cta_min, len(twc))
    assert np.array_equal(twc, exp * it)
    G.set_params(cta_stats=0)
    G.bfs(src, o)
    assert G.cta_loads()[0].size == 0
    G.close()


def test_hub_updates_aggregated_per_cta():
    """Hubs of degree > 2^16 take most updates (k-core combines its decrements to such targets
    per CTA in shared memory and applies them once per CTA and round). k-core, sssp, bfs and cc
    stay exact, for several k and sources, in the graph mode and in the host-loop mode, at the
    default threshold, with no vertex huge and with every vertex huge."""
    g = gg.rmat(17, 16 << 17, 31, symmetrize=True, weighted=True, n_hubs=6, hub_degree=100000)
    deg = np.diff(g.offsets.astype(np.int64))
    assert int((deg >= 1 << 16).sum()) >= 6
    G = make(g)
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    hub = int(np.argmax(deg))
    small = int(np.flatnonzero(deg == 3)[0])
    cc_ref = oracle.cc(g.n, g.offsets, g.indices)
    for params in (dict(), dict(exec_mode=1), dict(hub_threshold=1 << 40), dict(hub_threshold=0)):
        G.set_params(**{"hub_threshold": -1, "exec_mode": 0, **params})
        for k in (2, 16, 40):
            G.kcore(k, o)
            assert np.array_equal(host(o), oracle.kcore(g.n, g.offsets, g.indices, k)), (params, k)
        for src in (hub, small):
            G.sssp(src, o)
            assert np.array_equal(host(o), oracle.sssp(g.n, g.offsets, g.indices, g.weights, src)), (params, src)
            G.bfs(src, o)
            assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, src)), (params, src)
        G.cc(o)
        assert np.array_equal(host(o), cc_ref), params
    C = G.clone()
    C.sssp(hub, o)
    assert np.array_equal(host(o), oracle.sssp(g.n, g.offsets, g.indices, g.weights, hub))
    C.close()
    G.close()


def test_tile_push_overflow_goes_to_the_frontier():
    """A tile whose pushes exceed the CTA staging buffer (2048 entries): the centres of three
    stars of 3,000-6,000 leaves sit in the CTA bin (threshold above their degree), so one tile
    discovers thousands of vertices at once and the excess goes to the frontier directly. The
    leaves are chained so later rounds and k-core peeling have work too."""
    rng = np.random.Generator(np.random.Philox(key=11))
    n = 20000
    edges = []
    for c, lo, hi in ((0, 10, 6010), (1, 6010, 9010), (2, 9010, 14010)):
        edges += [(c, v) for v in range(lo, hi)]
    edges += [(0, 1), (1, 2)]
    edges += [(v, v + 1) for v in range(10, 14009)]
    edges += [(int(a), int(b)) for a, b in rng.integers(0, n, size=(20000, 2))]
    w = rng.integers(1, 101, size=len(edges))
    g = gg.from_edges(n, edges, w, symmetrize=True)
    G = make(g)
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for t in (1 << 40, -1, 100):
        G.set_params(hub_threshold=t)
        G.bfs(0, o)
        assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, 0)), t
        if t == 1 << 40:
            assert G.stats()["pushes"] > 3 * 2048  # the first BFS levels hold the three stars' leaves
        G.sssp(0, o)
        assert np.array_equal(host(o), oracle.sssp(g.n, g.offsets, g.indices, g.weights, 0)), t
        G.cc(o)
        assert np.array_equal(host(o), oracle.cc(g.n, g.offsets, g.indices)), t
        G.kcore(3, o)
        assert np.array_equal(host(o), oracle.kcore(g.n, g.offsets, g.indices, 3)), t
    G.close()


@pytest.mark.parametrize("frac", [0.25, 1.0])
def test_l2_persistence_window_keeps_results(rmat13, frac):
    """l2_persist_fraction > 0: the labels are computed in the handle's buffer under an L2
    access-policy window and copied out; results are unchanged, to device and host outputs."""
    g = rmat13
    src = g.max_degree_vertex()
    G = make(g)
    G.set_params(l2_persist_fraction=frac, hub_threshold=512)
    o = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.bfs(src, o)
    assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, src))
    G.sssp(src, o)
    assert np.array_equal(host(o), oracle.sssp(g.n, g.offsets, g.indices, g.weights, src))
    G.cc(o)
    assert np.array_equal(host(o), oracle.cc(g.n, g.offsets, g.indices))
    h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    G.kcore(3, h)
    G.sync()
    assert np.array_equal(h.numpy().view(np.uint32), oracle.kcore(g.n, g.offsets, g.indices, 3))
    G.close()


def test_batch_groups_run_concurrently_on_worker_clones(rmat13):
    """130 sources = five groups (the last ragged) dealt over the handle and three worker clones
    on their own streams; the same after a parameter change (the workers are rebuilt) and with
    the ragged group first in a second call of 33 sources."""
    g = rmat13
    G = make(g)
    rng = np.random.default_rng(21)
    srcs = rng.integers(0, g.n, size=130).astype(np.uint32)
    out = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    for params in (dict(), dict(hub_threshold=64), dict(exec_mode=1)):
        G.set_params(**{"hub_threshold": -1, "exec_mode": 0, **params})
        G.bfs_batch(srcs, out)
        lv = host(out).reshape(len(srcs), g.n).copy()
        G.sssp_batch(srcs, out)
        ds = host(out).reshape(len(srcs), g.n).copy()
        G.sync()
        for i in range(0, len(srcs), 7):
            s = int(srcs[i])
            assert np.array_equal(lv[i], oracle.bfs(g.n, g.offsets, g.indices, s)), (params, i)
            assert np.array_equal(ds[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, s)), (params, i)
        assert np.array_equal(lv[129], oracle.bfs(g.n, g.offsets, g.indices, int(srcs[129])))
    G.bfs_batch(srcs[:33], out)
    lv = host(out)[:33 * g.n].reshape(33, g.n)
    assert np.array_equal(lv[32], oracle.bfs(g.n, g.offsets, g.indices, int(srcs[32])))
    G.close()


def test_batch_worker_round_limit_reaches_sync():
    """A round limit hit only by a group that runs on a worker clone is reported by alb_sync of
    the handle: group 0 (on the handle) holds isolated vertices, group 1 (on a worker) walks a
    path longer than the limit."""
    n = 100
    g = gg.from_edges(n, [(v, v + 1) for v in range(40, 99)], symmetrize=True)
    G = make(g)
    G.set_params(max_rounds=5)
    srcs = np.array(list(range(32)) + [40], dtype=np.uint32)
    out = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
    G.bfs_batch(srcs, out)
    with pytest.raises(alb.AlbError) as e:
        G.sync()
    assert e.value.code == 4
    G.set_params(max_rounds=0)
    G.bfs_batch(srcs, out)
    G.sync()
    assert np.array_equal(host(out)[32 * n:33 * n], oracle.bfs(g.n, g.offsets, g.indices, 40))
    G.close()
