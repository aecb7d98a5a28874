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


# ----------------------------------------------------------- admission by free device memory
#
# The server's scheduling is independent of CUDA: a simulated device (a byte ledger behind
# mem_get_info) and a backend that allocates from it exercise admission, deferral and eviction.

class _Dev:
    def __init__(self, total):
        self.total, self.used, self.external = total, 0, 0
        self.min_free = total
        self.calls = 0
        self.release_external_after = None   # mem_get_info calls after which `external` drops

    def mem_get_info(self):
        self.calls += 1
        if self.release_external_after is not None and self.calls > self.release_external_after:
            self.external = 0
        return self.total - self.used - self.external, self.total

    def alloc(self, b):
        self.used += b
        self.min_free = min(self.min_free, self.total - self.used - self.external)


class _Buf:
    def __init__(self, dev, b):
        self.dev, self.b = dev, b
        dev.alloc(b)

    def __del__(self):
        self.dev.used -= self.b


class _G:
    def __init__(self, dev, b):
        self.dev, self.b, self.ws = dev, b, 0
        dev.alloc(b)


class _Ev:
    def __init__(self, polls):
        self.polls = polls


class FakeBackend:
    def __init__(self, dev, polls=2):
        self.dev, self.polls = dev, polls
        self.launches = []

    def sms(self, part): return 152
    def part_for(self, big): return None
    def mem_get_info(self): return self.dev.mem_get_info()
    def cached(self): return 0
    def priority_range(self): return (0, -1)
    def upload(self, csr, grid, tune_src): return _G(self.dev, serve.csr_bytes(csr) + serve.ROUND_WS_PER_VERTEX * csr.n)
    def clone(self, G):
        n = G.n
        c = _G(self.dev, serve.ROUND_WS_PER_VERTEX * n)
        c.n = n
        return c

    def destroy(self, G):
        self.dev.used -= G.b + G.ws
        G.b = G.ws = 0

    def trim(self, G):
        f = G.ws
        self.dev.used -= f
        G.ws = 0
        return f

    def stream(self, priority, part): return object()
    def buffers(self, n, kind): return (_Buf(self.dev, serve.result_bytes(n, kind)), None)
    def source_buffer(self): return [0] * (2 * serve.GROUP)

    def warm(self, slot, kinds, src):
        if any(k in ("bfs", "sssp") for k in kinds) and slot.G.ws == 0:
            slot.G.ws = serve.BATCH_WS_PER_VERTEX * slot.n
            self.dev.alloc(slot.G.ws)

    def launch(self, slot, bq, sq, cq):
        self.launches.append([r.rid for r in bq + sq + cq])
        return _Ev(self.polls)

    def done(self, ev):
        ev.polls -= 1
        return ev.polls <= 0

    def result(self, slot, kind, j): return np.zeros(1, dtype=np.uint32)
    def check(self, slot): pass
    def synchronize(self): pass
    def release_buffers(self): pass
    def close(self): pass


def _fake_server(graphs, total, reserve, **kw):
    dev = _Dev(total)
    be = FakeBackend(dev)
    orig_upload = be.upload

    def upload(csr, grid, tune_src):
        G = orig_upload(csr, grid, tune_src)
        G.n = csr.n
        return G
    be.upload = upload
    srv = serve.Server(graphs, tune=False, backend=be, hbm_reserve=reserve, **kw)
    return srv, dev, be


def _full_need(g):
    return (serve.csr_bytes(g) + serve.ROUND_WS_PER_VERTEX * g.n + sum(serve.result_bytes(g.n, k) for k in serve.KINDS)
            + serve.BATCH_WS_PER_VERTEX * g.n)


def _in_arrival_order(srv, reqs):
    by = {}
    for gid, kind, rid in srv.admit_log:
        by.setdefault((gid, kind), []).append(rid)
    return all(v == sorted(v) for v in by.values()) and sum(map(len, by.values())) == len(reqs)


def test_batches_wait_for_free_memory_then_run_in_arrival_order():
    gs = _graphs()
    reserve = 1 << 20
    total = reserve + _full_need(gs[0]) + 4096
    srv, dev, be = _fake_server(gs[:1], total, reserve, lazy=True)
    dev.external = total            # another user of the device holds everything at first
    dev.release_external_after = 40
    reqs = serve.poisson_requests(gs[:1], 80, rate=1e6, seed=7)
    srv.run(reqs, realtime=False, timeout=30)
    assert all(r.done >= 0 for r in reqs)
    assert srv.deferred >= 1                       # refused while the memory was taken
    assert _in_arrival_order(srv, reqs)            # and admitted in order afterwards
    assert dev.min_free >= reserve                 # nothing was admitted below the reserve


def test_graphs_are_evicted_and_readmitted_when_memory_is_short():
    """Room for one graph with all its buffers plus half of another graph's CSR: requests for
    graph 0, then graph 1, then graph 0 again. Graph 0 is evicted (idle, nothing queued) to
    admit graph 1, and uploaded again for its second wave."""
    gs = [gg.rmat(10, 16 << 10, 600 + i, symmetrize=True, weighted=True) for i in range(2)]
    reserve = 1 << 20
    up = max(serve.csr_bytes(g) + serve.ROUND_WS_PER_VERTEX * g.n for g in gs)
    total = reserve + max(_full_need(g) for g in gs) + up // 2
    srv, dev, be = _fake_server(gs, total, reserve, lazy=True)
    kinds = serve.KINDS
    reqs = [serve.Request(i, 0.05 * (i // 40), (i // 40) % 2, kinds[i % 3], 1 + i % 11) for i in range(120)]
    srv.run(reqs, realtime=True, timeout=30)
    assert all(r.done >= 0 for r in reqs)
    assert srv.evictions > 0                       # idle resources gave their memory back
    assert srv.graphs[0].uploads == 2              # graph 0 was evicted and uploaded again
    assert _in_arrival_order(srv, reqs)
    assert dev.min_free >= reserve


def test_an_extra_slot_is_admitted_while_memory_allows():
    g = gg.rmat(10, 16 << 10, 3, symmetrize=True, weighted=True)
    reserve = 1 << 20
    srv, dev, be = _fake_server([g], reserve + 4 * _full_need(g), reserve, lazy=True,
                                big_graph_edges=1, big_slots=2)
    reqs = [serve.Request(i, 0.0, 0, "bfs", 1 + i % 7) for i in range(96)]
    srv.run(reqs, realtime=False, timeout=30)
    assert srv.admitted_slots == 1 and len(srv.graphs[0].slots) == 2
    assert all(r.done >= 0 for r in reqs)
    # with no room for a clone, the graph keeps one slot
    srv2, dev2, _ = _fake_server([g], reserve + _full_need(g) + 1024, reserve, lazy=True,
                                 big_graph_edges=1, big_slots=2)
    reqs = [serve.Request(i, 0.0, 0, "bfs", 1 + i % 7) for i in range(96)]
    srv2.run(reqs, realtime=False, timeout=30)
    assert srv2.admitted_slots == 0 and len(srv2.graphs[0].slots) == 1
    assert all(r.done >= 0 for r in reqs)


def test_batch_bytes_count_only_what_the_slot_lacks():
    g = gg.rmat(8, 16 << 8, 3, symmetrize=True, weighted=True)
    srv, dev, be = _fake_server([g], 1 << 40, 0, lazy=True)
    srv._admit_graph(srv.graphs[0])
    gr = srv.graphs[0]
    s = gr.slots[0]
    n = g.n
    assert gr.batch_bytes(s, 3, 0, 0) == 4 * 32 * n + serve.BATCH_WS_PER_VERTEX * n
    assert gr.batch_bytes(s, 0, 0, 2) == 4 * n
    s.ensure(["bfs"], 0)
    assert gr.batch_bytes(s, 3, 0, 0) == 0
    assert gr.batch_bytes(s, 0, 5, 0) == 4 * 32 * n          # the batch workspace is shared
    assert gr.batch_bytes(s, 1, 1, 1) == 4 * 32 * n + 4 * n
