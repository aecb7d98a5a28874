"""Continuous-batching server: every result is the same alone and in the mix."""
import numpy as np
import pytest

import oracle
from paper_1911_09135_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_09135_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module")
def graphs():
    return [gg.rmat(sc, 16 << sc, 500 + i, symmetrize=True, weighted=True)
            for i, sc in enumerate((8, 10, 11, 13))]


@pytest.mark.parametrize("small_sms", [0, 16])
def test_results_alone_equal_results_in_the_mix(graphs, small_sms):
    """Also with the small graphs on an SM partition of their own (small_sms > 0)."""
    reqs = serve.poisson_requests(graphs, 400, rate=20000.0, seed=5)
    srv = serve.Server(graphs, tune=False, keep_results=True, big_graph_edges=100_000,
                       small_sms=small_sms)
    try:
        assert len(srv.graphs[-1].slots) == 2            # a large graph gets a second slot (a clone)
        srv.run(reqs, realtime=True, timeout=120)
        assert all(r.done >= r.arrival for r in reqs)
        assert srv.batches < len(reqs)               # requests were batched together
        _, alone = serve.one_at_a_time(srv, reqs, keep_results=True)
    finally:
        srv.close()
    for r in reqs:
        assert np.array_equal(srv.results[r.rid], alone[r.rid]), (r.rid, r.kind)
    # and a sample against the oracle
    for r in reqs[:30]:
        g = graphs[r.graph]
        if r.kind == "bfs":
            ref = oracle.bfs(g.n, g.offsets, g.indices, r.src)
        elif r.kind == "sssp":
            ref = oracle.sssp(g.n, g.offsets, g.indices, g.weights, r.src)
        else:
            ref = oracle.cc(g.n, g.offsets, g.indices)
        assert np.array_equal(srv.results[r.rid], ref), (r.rid, r.kind)


def test_config5_large_graphs_alone_equal_mix_equal_oracle():
    """The two largest serving graphs that fit the test budget (RMAT scales 20 and 21, seeds 504
    and 505, as in the 8-graph serving mix), a short Poisson mix at 2,000 requests/s: every
    served result equals the same request run alone, and a sample of each kind equals the
    oracle."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    big = [gg.rmat(sc, 16 << sc, 500 + i, symmetrize=True, weighted=True)
           for i, sc in ((4, 20), (5, 21))]
    reqs = serve.poisson_requests(big, 240, rate=2000.0, seed=5)
    srv = serve.Server(big, tune=False, keep_results=True)
    try:
        assert len(srv.graphs[-1].slots) == 2        # m >= 50M: the larger graph has two slots
        srv.run(reqs, realtime=True, timeout=300)
        assert all(r.done >= r.arrival for r in reqs)
        assert srv.batches < len(reqs)
        _, alone = serve.one_at_a_time(srv, reqs, keep_results=True)
    finally:
        srv.close()
    for r in reqs:
        assert np.array_equal(srv.results[r.rid], alone[r.rid]), (r.rid, r.kind)
    sample = []
    for kind in serve.KINDS:
        for gi in range(len(big)):
            sample += [r for r in reqs if r.kind == kind and r.graph == gi][:2]

    def ref(r):
        g = big[r.graph]
        if r.kind == "bfs":
            return oracle.bfs(g.n, g.offsets, g.indices, r.src)
        if r.kind == "sssp":
            return oracle.sssp(g.n, g.offsets, g.indices, g.weights, r.src)
        return oracle.cc(g.n, g.offsets, g.indices)

    with ThreadPoolExecutor(max_workers=len(os.sched_getaffinity(0))) as ex:
        refs = list(ex.map(ref, sample))
    assert len(sample) >= 10
    for r, want in zip(sample, refs):
        assert np.array_equal(srv.results[r.rid], want), (r.rid, r.kind, r.graph)


def test_lazy_slots_wait_for_free_device_memory_then_serve_in_order(graphs):
    """Slots set up on first use (lazy): the free memory the server sees is held below what the
    first batches need for a while (an injected cudaMemGetInfo: another user of the device), so
    they are deferred and stay queued; once memory frees up they are admitted in arrival order,
    their buffers and workspaces are set up, and every result equals the oracle."""
    real = torch.cuda.mem_get_info
    calls = {"n": 0}

    def squeezed():
        calls["n"] += 1
        free, total = real()
        return (0 if calls["n"] <= 50 else free), total

    reqs = serve.poisson_requests(graphs, 60, rate=1e6, seed=6)
    srv = serve.Server(graphs, tune=False, keep_results=True, lazy=True, mem_get_info=squeezed,
                       hbm_reserve=1 << 28)
    try:
        srv.run(reqs, realtime=False, timeout=120)
    finally:
        srv.close()
    assert srv.deferred >= 1 and all(r.done >= 0 for r in reqs)
    by = {}
    for gid, kind, rid in srv.admit_log:
        by.setdefault((gid, kind), []).append(rid)
    assert all(v == sorted(v) for v in by.values())
    for r in reqs:
        g = graphs[r.graph]
        if r.kind == "bfs":
            ref = oracle.bfs(g.n, g.offsets, g.indices, r.src)
        elif r.kind == "sssp":
            ref = oracle.sssp(g.n, g.offsets, g.indices, g.weights, r.src)
        else:
            ref = oracle.cc(g.n, g.offsets, g.indices)
        assert np.array_equal(srv.results[r.rid], ref), (r.rid, r.kind)


def test_sm_partition_streams_run_the_library_exactly(graphs):
    """Streams of both halves of an SM split run every app exactly (kernels, CUDA graphs with
    device-side loops); the halves cover the device."""
    from paper_1911_09135_gb300 import alb
    first, rest = alb.partition_split(torch.cuda.current_device(), 16)
    try:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        assert first.sms >= 16 and first.sms + rest.sms == sms
        g = graphs[-1]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
        G = alb.Graph(g.n, dev(g.offsets), dev(g.indices), dev(g.weights), symmetric=True)
        o = torch.empty(g.n, dtype=torch.int32, device="cuda")
        src = g.max_degree_vertex()
        for part in (first, rest):
            s = torch.cuda.ExternalStream(part.stream())
            with torch.cuda.stream(s):
                alb.alb_bfs(G.h, src, o, s)
                s.synchronize()
                assert np.array_equal(o.cpu().numpy().view(np.uint32), oracle.bfs(g.n, g.offsets, g.indices, src))
                alb.alb_sssp(G.h, src, o, s)
                s.synchronize()
                assert np.array_equal(o.cpu().numpy().view(np.uint32),
                                      oracle.sssp(g.n, g.offsets, g.indices, g.weights, src))
        G.close()
    finally:
        torch.cuda.synchronize()
        first.close()
        rest.close()


def test_sm_partition_argument_errors():
    from paper_1911_09135_gb300 import alb
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for bad in (0, sms, sms + 8):
        with pytest.raises(alb.AlbError) as e:
            alb.partition_split(torch.cuda.current_device(), bad)
        assert e.value.code == 1  # ALB_ERR_INVALID_ARG: nothing is created
    first, rest = alb.partition_split(torch.cuda.current_device(), 1)   # rounded up to the granularity
    try:
        assert first.sms >= 1 and first.sms % 8 == 0 and first.sms + rest.sms == sms
    finally:
        first.close()
        rest.close()


def test_trim_releases_workspaces_and_the_handle_stays_exact():
    """alb_graph_trim gives back what the handle's calls allocated on first use (batch workspace,
    cached CUDA graphs, PageRank's vectors) and the next calls set them up again, exactly."""
    from paper_1911_09135_gb300 import alb
    g = gg.rmat(16, 16 << 16, 77, symmetrize=True, weighted=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    G = alb.Graph(g.n, dev(g.offsets), dev(g.indices), dev(g.weights), symmetric=True)
    try:
        srcs = np.array([0, 5, g.max_degree_vertex()], dtype=np.uint32)
        out = torch.empty(3 * g.n, dtype=torch.int32, device="cuda")
        r = torch.empty(g.n, dtype=torch.float32, device="cuda")
        for rep in range(2):
            G.sssp_batch(srcs, out)
            G.pagerank(0.85, 1e-6, 1000, r)
            G.sync()
            got = out.cpu().numpy().view(np.uint32).reshape(3, g.n)
            for i, s in enumerate(srcs.tolist()):
                assert np.array_equal(got[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, s)), (rep, i)
            if rep == 0:
                torch.cuda.synchronize()
                freed = G.trim()
                # the multi-source workspace alone is 144 bytes per vertex (9.4 MB here); the
                # device reports free memory in whole pages, so compare with half of it
                assert freed >= 72 * g.n, freed
    finally:
        G.close()


def test_eviction_and_reupload_on_the_gpu():
    """Lazy serving under a memory budget that holds one graph with its buffers: requests for
    graph 0, then graph 1, then graph 0 again make the server evict idle resources (buffers,
    cached workspaces through alb_graph_trim, whole graphs) and upload graph 0 again; every result
    equals the oracle. The free memory the server sees is its own account of what it holds
    (graphs, slots, buffers, workspaces) under the budget."""
    gs = [gg.rmat(12, 16 << 12, 610 + i, symmetrize=True, weighted=True) for i in range(2)]
    full = max(serve.csr_bytes(g) + serve.ROUND_WS_PER_VERTEX * g.n
               + sum(serve.result_bytes(g.n, k) for k in serve.KINDS) + serve.BATCH_WS_PER_VERTEX * g.n
               for g in gs)
    up = max(serve.csr_bytes(g) + serve.ROUND_WS_PER_VERTEX * g.n for g in gs)
    budget = full + up // 2
    holder = {}

    def held():
        srv = holder["srv"]
        used = 0
        for gr in srv.graphs:
            if not gr.resident:
                continue
            used += gr.upload_bytes() + gr.clone_bytes() * (len(gr.slots) - 1)
            for s in gr.slots:
                used += sum(serve.result_bytes(s.n, k) for k in s.bufs)
                if s.warmed & {"bfs", "sssp"}:
                    used += serve.BATCH_WS_PER_VERTEX * s.n
        return budget - used, budget

    srv = serve.Server(gs, tune=False, keep_results=True, lazy=True, hbm_reserve=0,
                       mem_get_info=lambda: held())
    holder["srv"] = srv
    kinds = serve.KINDS
    reqs = [serve.Request(i, 0.05 * (i // 30), (i // 30) % 2, kinds[i % 3], 1 + (i * 37) % 4000)
            for i in range(90)]
    try:
        srv.run(reqs, realtime=True, timeout=120)
    finally:
        srv.close()
    assert srv.evictions > 0 and srv.graphs[0].uploads == 2
    for r in reqs:
        g = gs[r.graph]
        if r.kind == "bfs":
            ref = oracle.bfs(g.n, g.offsets, g.indices, r.src)
        elif r.kind == "sssp":
            ref = oracle.sssp(g.n, g.offsets, g.indices, g.weights, r.src)
        else:
            ref = oracle.cc(g.n, g.offsets, g.indices)
        assert np.array_equal(srv.results[r.rid], ref), (r.rid, r.kind, r.graph)
