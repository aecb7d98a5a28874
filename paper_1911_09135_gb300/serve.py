"""Continuous-batching query server over resident graphs (bfs / sssp / cc).

Graphs are uploaded once and stay resident. Each has one or more slots (a handle with its own
CUDA stream; extra slots are clones sharing the graph's device CSR, given to large graphs).
Smaller graphs run on higher-priority streams, and every slot's grid is sized to its graph
(at most two CTAs per SM), so kernels of several slots share the SMs. Requests arrive open-loop; each is queued
on its graph. Whenever one of a graph's slots is idle
and queued work exists, the server forms one batch from that graph's queue - up to 32 bfs sources and 32 sssp
sources (one multi-source group each, sharing every CSR read: alb_bfs_batch / alb_sssp_batch)
plus every queued cc query (one alb_cc serves them all), launches it on the slot's stream and
copies the requested rows to pinned host memory. Device memory is admitted per slot: a slot
(its result buffers and workspaces) is created only if free HBM covers it, and no batch is
launched while free HBM is below a reserve (memory taken by other users of the GPU); the
slots' buffers are allocated up front, so nothing is allocated while kernels run. Slots of different graphs run concurrently on the device, and requests that
arrive meanwhile wait for the next batch of their graph. A request's latency runs from its
arrival to the completion of its result's device-to-host copy.

All traversal work runs in libalb.so; this module only schedules calls.

The device multiplexes streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware work queues (8 by
default): slots whose streams share a queue run in its FIFO order, so a small graph's batch waits
behind a large graph's. A serving process sets CUDA_DEVICE_MAX_CONNECTIONS=32 before CUDA starts
(the server warns when it has more slots than queues). `small_sms` instead gives the small graphs
an SM partition of their own (a green context, alb_partition_split); it is off by default: with
enough queues the SMs are shared well, and a fixed partition measured slower.
"""
from __future__ import annotations

import dataclasses
import os
import time
from collections import deque

import numpy as np

from . import alb

GROUP = 32
KINDS = ("bfs", "sssp", "cc")
EDGES_PER_CTA = 1 << 17       # serving grids: one CTA per this many edges, at most ctas_per_sm per SM


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float   # seconds from the start of the run
    graph: int
    kind: str        # "bfs" | "sssp" | "cc"
    src: int = 0
    done: float = -1.0


def poisson_requests(graphs, count: int, rate: float, seed: int = 5) -> list[Request]:
    """Open-loop Poisson arrivals (rate per second); graph and kind uniform; source uniform over
    the graph's non-isolated vertices."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    gi = rng.integers(0, len(graphs), size=count)
    ki = rng.integers(0, len(KINDS), size=count)
    nonisolated = [np.nonzero(g.degrees() > 0)[0] for g in graphs]
    out = []
    for i in range(count):
        cand = nonisolated[gi[i]]
        src = int(cand[rng.integers(0, len(cand))]) if len(cand) else 0
        out.append(Request(i, float(t[i]), int(gi[i]), KINDS[ki[i]], src))
    return out


class _Slot:
    """One handle (the graph's own, or a clone sharing its CSR) with its stream and buffers."""

    def __init__(self, torch, G, n, priority: int, part=None):
        self.G = G
        self.n = n
        # a stream of the graph's SM partition, else an ordinary one
        self.stream = (torch.cuda.ExternalStream(part.stream(priority)) if part is not None
                       else torch.cuda.Stream(priority=priority))
        self.busy = None      # (event, batch info) while a batch is in flight
        # Result buffers of one batch, allocated once: nothing is allocated while other slots'
        # kernels run (an allocation can wait for the whole device).
        self.d_bfs = torch.empty(GROUP * n, dtype=torch.int32, device="cuda")
        self.d_sssp = torch.empty(GROUP * n, dtype=torch.int32, device="cuda")
        self.d_cc = torch.empty(n, dtype=torch.int32, device="cuda")
        self.h_bfs = torch.empty(GROUP * n, dtype=torch.int32).pin_memory()
        self.h_sssp = torch.empty(GROUP * n, dtype=torch.int32).pin_memory()
        self.h_cc = torch.empty(n, dtype=torch.int32).pin_memory()
        self.h_srcs = torch.empty(2 * GROUP, dtype=torch.int32).pin_memory()

    def warm(self, src: int):
        """First use of every call on this slot (workspace allocation, graph instantiation)."""
        self.h_srcs[0] = src
        self.h_srcs[GROUP] = src
        alb.alb_bfs_batch(self.G.h, self.h_srcs[:1], 1, self.d_bfs, self.stream)
        alb.alb_sssp_batch(self.G.h, self.h_srcs[GROUP:GROUP + 1], 1, self.d_sssp, self.stream)
        alb.alb_cc(self.G.h, self.d_cc, self.stream)
        self.stream.synchronize()


class _Graph:
    """A resident graph: its request queues and one or more slots."""

    @staticmethod
    def slot_bytes(n: int) -> int:
        """Device memory one slot holds: result buffers (2 x 32 labels + 1 per vertex), the
        multi-source workspace (148 bytes per vertex) and the round workspace (20 per vertex)."""
        return n * (4 * (2 * GROUP + 1) + 148 + 20)

    def __init__(self, torch, csr, tune: bool, slots: int, priority: int, ctas_per_sm: int = 2,
                 part=None):
        self.n = csr.n
        self.m = csr.m
        self.deg = csr.degrees().astype(np.int64)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
        G = alb.Graph(csr.n, dev(csr.offsets), dev(csr.indices), dev(csr.weights),
                      symmetric=csr.symmetric)
        # A persistent grid over the whole GPU would keep other slots' kernels waiting until it
        # ends: small graphs get a grid sized to their edges, large ones two CTAs per SM, so
        # kernels of several slots share the SMs.
        sms = (part.sms if part is not None else
               torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
        G.set_params(grid_blocks=min(ctas_per_sm * sms, max(16, -(-csr.m // EDGES_PER_CTA))))
        if tune:
            src = int(np.argmax(self.deg))
            for k in KINDS:
                G.autotune(k, src, reps=1)
        handles = [G]
        for _ in range(slots - 1):  # extra slots only while free device memory allows
            free, _ = torch.cuda.mem_get_info()
            if free < 2 * self.slot_bytes(csr.n) + (1 << 30):
                break
            handles.append(G.clone())  # clones keep the tuned knobs
        self.slots = [_Slot(torch, h, csr.n, priority, part) for h in handles]
        for sl in self.slots:
            sl.warm(int(np.argmax(self.deg)))
        self.queue = {k: deque() for k in KINDS}
        self.log = []         # (seconds in flight, #bfs, #sssp, #cc) per completed batch

    def batch_bytes(self, nb, ns, nc) -> int:
        # result buffers are allocated with the slot; a batch needs no further device memory
        return 0

    def close(self):
        for s in reversed(self.slots):
            s.G.close()


class Server:
    """One slot per resident graph; see the module docstring."""

    def __init__(self, graphs, *, tune: bool = True, keep_results: bool = False,
                 hbm_reserve: int = 1 << 30, big_graph_edges: int = 50_000_000, big_slots: int = 2,
                 ctas_per_sm: int = 2, small_sms: int = 0):
        import torch
        self.torch = torch
        # small_sms > 0: the graphs below big_graph_edges get an SM partition of that many SMs and
        # the large graphs the rest, so small graphs' round kernels never wait for SM room held
        # by the large graphs' persistent kernels
        self.parts = None
        if small_sms > 0:
            self.parts = alb.partition_split(torch.cuda.current_device(), small_sms)
        # smaller graphs get higher stream priority, so their short rounds are scheduled
        # between the round kernels of large graphs instead of waiting behind them
        lo, hi = torch.cuda.Stream.priority_range()
        order = np.argsort(np.argsort([g.m for g in graphs]))
        prio = [hi if order[i] < len(graphs) // 2 else lo for i in range(len(graphs))]
        def part_of(g):
            if self.parts is None:
                return None
            return self.parts[1] if g.m >= big_graph_edges else self.parts[0]
        self.graphs = [_Graph(torch, g, tune, big_slots if g.m >= big_graph_edges else 1, prio[i], ctas_per_sm,
                              part_of(g))
                       for i, g in enumerate(graphs)]
        slots = sum(len(g.slots) for g in self.graphs)
        queues = int(os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"))
        if slots + 1 > queues:
            import warnings
            warnings.warn(f"{slots} slot streams share {queues} hardware work queues; set "
                          f"CUDA_DEVICE_MAX_CONNECTIONS={min(32, slots + 1)} before CUDA starts")
        self.keep = keep_results
        self.reserve = hbm_reserve
        self.results: dict[int, np.ndarray] = {}
        self.batches = 0
        self.deferred = 0     # batch formations postponed for lack of free device memory
        self.edges = 0        # traversed-edge units of completed requests (m of the graph each)
        # with the bounds-checked library, every completed batch's record is inspected
        self.checked = os.environ.get("ALB_CHECKED") == "1" and alb.alb_checked_build() == 1

    def close(self):
        torch = self.torch
        torch.cuda.synchronize()
        for g in self.graphs:
            g.close()
        if self.parts is not None:
            # the partitions' streams go last: first the buffers used on them, and the blocks the
            # caching allocator may still associate with them
            for g in self.graphs:
                g.slots = []
            import gc
            gc.collect()
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            for p in self.parts:
                p.close()
            self.parts = None

    def _free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info()
        cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        return int(free + cached)

    def _launch(self, gr: _Graph, s: _Slot):
        torch = self.torch
        bq = [gr.queue["bfs"].popleft() for _ in range(min(GROUP, len(gr.queue["bfs"])))]
        sq = [gr.queue["sssp"].popleft() for _ in range(min(GROUP, len(gr.queue["sssp"])))]
        cq = list(gr.queue["cc"])
        gr.queue["cc"].clear()
        need = gr.batch_bytes(len(bq), len(sq), len(cq))
        if self._free_bytes() - need < self.reserve:
            # not admitted: back to the front of the queues, retried when memory frees up
            for q, items in (("bfs", bq), ("sssp", sq), ("cc", cq)):
                gr.queue[q].extendleft(reversed(items))
            self.deferred += 1
            return False
        n = s.n
        # the slot's pinned source list is free: its previous batch has completed
        for j, r in enumerate(bq):
            s.h_srcs[j] = r.src
        for j, r in enumerate(sq):
            s.h_srcs[GROUP + j] = r.src
        with torch.cuda.stream(s.stream):
            if bq:
                alb.alb_bfs_batch(s.G.h, s.h_srcs[:len(bq)], len(bq), s.d_bfs, s.stream)
                s.h_bfs[: len(bq) * n].copy_(s.d_bfs[: len(bq) * n], non_blocking=True)
            if sq:
                alb.alb_sssp_batch(s.G.h, s.h_srcs[GROUP:GROUP + len(sq)], len(sq), s.d_sssp, s.stream)
                s.h_sssp[: len(sq) * n].copy_(s.d_sssp[: len(sq) * n], non_blocking=True)
            if cq:
                alb.alb_cc(s.G.h, s.d_cc, s.stream)
                s.h_cc.copy_(s.d_cc, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s.stream)
        s.busy = (ev, bq, sq, cq, None, time.perf_counter())
        self.batches += 1
        return True

    def _complete(self, gr: _Graph, s: _Slot, now: float):
        ev, bq, sq, cq, bufs, t_launch = s.busy
        if self.checked:
            rec = alb.alb_debug_check(s.G.h)
            if rec[0]:
                raise RuntimeError(f"bounds check failed on graph n={gr.n} m={gr.m} slot "
                                   f"{gr.slots.index(s)}: code {rec[0]} index {rec[1]} bound {rec[2]} "
                                   f"count {rec[3]}; batch bfs={len(bq)} sssp={len(sq)} cc={len(cq)}")
        gr.log.append((time.perf_counter() - t_launch, len(bq), len(sq), len(cq)))
        n = s.n
        self.edges += gr.m * (len(bq) + len(sq) + len(cq))
        for j, r in enumerate(bq):
            r.done = now
            if self.keep:
                self.results[r.rid] = s.h_bfs[j * n:(j + 1) * n].numpy().view(np.uint32).copy()
        for j, r in enumerate(sq):
            r.done = now
            if self.keep:
                self.results[r.rid] = s.h_sssp[j * n:(j + 1) * n].numpy().view(np.uint32).copy()
        for r in cq:
            r.done = now
            if self.keep:
                self.results[r.rid] = s.h_cc.numpy().view(np.uint32).copy()
        s.busy = None

    def run(self, requests: list[Request], *, realtime: bool = True, timeout: float = 600.0):
        """Serve `requests` (sorted by arrival). realtime=False admits everything at once
        (saturation throughput). Returns wall seconds from the first arrival to the last result."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        i, pending = 0, len(reqs)
        while pending:
            now = time.perf_counter() - t0
            if now > timeout:
                raise TimeoutError("serving run exceeded its time limit")
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                r = reqs[i]
                if not realtime:
                    r.arrival = 0.0
                self.graphs[r.graph].queue[r.kind].append(r)
                i += 1
            progressed = False
            for gr in self.graphs:
                for s in gr.slots:
                    if s.busy is not None and s.busy[0].query():
                        before = sum(len(x) for x in s.busy[1:4])
                        self._complete(gr, s, time.perf_counter() - t0)
                        pending -= before
                        progressed = True
                    if s.busy is None and any(gr.queue[k] for k in KINDS):
                        progressed |= self._launch(gr, s)
            if not progressed:
                time.sleep(0.0001)
        return time.perf_counter() - t0


def one_at_a_time(graphs_or_server, requests: list[Request], *, keep_results: bool = False):
    """Reference path: one request at a time, in arrival order, each with its own call on one
    stream (alb_bfs / alb_sssp / alb_cc), results copied to the host. Returns (seconds, results)."""
    srv = graphs_or_server
    torch = srv.torch
    res = {}
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        s = srv.graphs[r.graph].slots[0]
        out = torch.empty(s.n, dtype=torch.int32, device="cuda")
        if r.kind == "bfs":
            alb.alb_bfs(s.G.h, r.src, out)
        elif r.kind == "sssp":
            alb.alb_sssp(s.G.h, r.src, out)
        else:
            alb.alb_cc(s.G.h, out)
        h = out.cpu()
        if keep_results:
            res[r.rid] = h.numpy().view(np.uint32).copy()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, res


def slot_stats(server: "Server", requests: list[Request]) -> list[dict]:
    """Per graph: latency percentiles, batches, mean batch time and size."""
    out = []
    for gi, s in enumerate(server.graphs):
        rs = [r for r in requests if r.graph == gi]
        lat = np.array([r.done - r.arrival for r in rs]) * 1e3 if rs else np.zeros(1)
        log = np.array(s.log) if s.log else np.zeros((1, 4))
        out.append({"graph": gi, "m": s.m, "slots": len(s.slots), "requests": len(rs),
                    "p50_ms": round(float(np.percentile(lat, 50)), 2),
                    "p99_ms": round(float(np.percentile(lat, 99)), 2),
                    "batches": len(s.log), "batch_ms_mean": round(float(log[:, 0].mean() * 1e3), 2),
                    "batch_size_mean": round(float(log[:, 1:].sum(axis=1).mean()), 1)})
    return out


def latency_stats(requests: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in requests], dtype=np.float64) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "max_ms": round(float(lat.max()), 3)}
