"""Continuous-batching query server over resident graphs (bfs / sssp / cc).

Graphs are uploaded once and stay resident while device memory allows. Each has one or more
slots (a handle with its own CUDA stream; extra slots are clones sharing the graph's device CSR,
given to large graphs). Smaller graphs run on higher-priority streams, and every slot's grid is
sized to its graph (at most two CTAs per SM), so kernels of several slots share the SMs. Requests
arrive open-loop; each is queued on its graph. Whenever one of a graph's slots is idle and queued
work exists, the server forms one batch from that graph's queue - up to 32 bfs sources and 32
sssp sources (one multi-source group each, sharing every CSR read: alb_bfs_batch /
alb_sssp_batch) plus every queued cc query (one alb_cc serves them all), launches it on the
slot's stream and copies the requested rows to pinned host memory. Slots of different graphs
run concurrently on the device, and requests that arrive meanwhile wait for the next batch of
their graph. A request's latency runs from its arrival to the completion of its result's
device-to-host copy.

Device memory is admitted by free HBM (cudaMemGetInfo plus the caching allocator's idle blocks):
  - a graph is uploaded (its CSR and round workspace), a slot is created (a clone's round
    workspace), and a batch gets whatever its slot still lacks (result buffers of its kinds and
    the library's multi-source workspace) only if the free memory stays above a reserve
    afterwards;
  - a batch that does not fit goes back to the front of its graph's queues (arrival order is
    kept) and is retried when memory frees up;
  - to make room, idle resources of other graphs are evicted, least recently used first: an
    extra slot (its clone and buffers), then a slot's result buffers and its handle's cached
    workspaces (alb_graph_trim), then, for graphs with nothing queued, the whole graph; an evicted
    graph is uploaded again when a request for it arrives.
By default every graph and slot is set up and warmed before serving, so a run that fits never
allocates while kernels run (set-up waits for an idle device); `lazy=True` defers all of it to
first use.

All traversal work runs in libalb.so; this module only schedules calls. The scheduling logic is
independent of CUDA: it talks to a backend (`CudaBackend` by default), so its admission and
eviction rules are testable on the host with a simulated device.

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

GROUP = 32
KINDS = ("bfs", "sssp", "cc")
EDGES_PER_CTA = 1 << 17       # serving grids: one CTA per this many edges, at most ctas_per_sm per SM

# Device bytes per vertex of the library's workspaces (include/alb.h): the round workspace of a
# handle (two frontiers, huge worklist and prefix, two push bitmaps) and the multi-source batch
# workspace (32 labels, a seen mask and three round masks per vertex).
ROUND_WS_PER_VERTEX = 17
BATCH_WS_PER_VERTEX = 144


def result_bytes(n: int, kind: str) -> int:
    """Device result buffer of one batch of `kind` on an n-vertex graph."""
    return 4 * n * (GROUP if kind in ("bfs", "sssp") else 1)


def csr_bytes(csr) -> int:
    return 4 * (csr.n + 1) + 4 * csr.m * (2 if csr.weights is not None else 1)


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


class Admission:
    """Free-HBM admission: `need` more bytes are admitted only if the device's free memory stays
    at or above `reserve` afterwards. `mem_get_info` returns (free, total) like
    cudaMemGetInfo; `cached` returns idle bytes a caching allocator holds (usable too)."""

    def __init__(self, mem_get_info, reserve: int, cached=None):
        self.mem_get_info = mem_get_info
        self.reserve = int(reserve)
        self.cached = cached or (lambda: 0)

    def free(self) -> int:
        free, _ = self.mem_get_info()
        return int(free) + int(self.cached())

    def admits(self, need: int) -> bool:
        return self.free() - int(need) >= self.reserve


class CudaBackend:
    """The device side of the server: libalb.so handles, torch streams, buffers and events."""

    def __init__(self, small_sms: int = 0):
        import torch

        from . import alb
        self.torch, self.alb = torch, alb
        self.parts = None
        if small_sms > 0:
            self.parts = alb.partition_split(torch.cuda.current_device(), small_sms)
        self.checked = os.environ.get("ALB_CHECKED") == "1" and alb.alb_checked_build() == 1

    def sms(self, part) -> int:
        if part is not None:
            return part.sms
        t = self.torch
        return t.cuda.get_device_properties(t.cuda.current_device()).multi_processor_count

    def part_for(self, big: bool):
        if self.parts is None:
            return None
        return self.parts[1] if big else self.parts[0]

    def mem_get_info(self):
        return self.torch.cuda.mem_get_info()

    def cached(self) -> int:
        t = self.torch
        return int(t.cuda.memory_reserved() - t.cuda.memory_allocated())

    def priority_range(self):
        return self.torch.cuda.Stream.priority_range()

    def upload(self, csr, grid_blocks: int, tune_src):
        t = self.torch
        dev = lambda a: t.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
        G = self.alb.Graph(csr.n, dev(csr.offsets), dev(csr.indices), dev(csr.weights),
                           symmetric=csr.symmetric)
        G.set_params(grid_blocks=grid_blocks)
        if tune_src is not None:
            for k in KINDS:
                G.autotune(k, tune_src, reps=1)
        return G

    def clone(self, G):
        return G.clone()  # clones keep the tuned knobs

    def destroy(self, G) -> None:
        G.close()

    def trim(self, G) -> int:
        return G.trim()

    def stream(self, priority: int, part):
        t = self.torch
        return (t.cuda.ExternalStream(part.stream(priority)) if part is not None
                else t.cuda.Stream(priority=priority))

    def buffers(self, n: int, kind: str):
        """(device, pinned host) result buffers of one batch of `kind`."""
        t = self.torch
        cnt = GROUP * n if kind in ("bfs", "sssp") else n
        return (t.empty(cnt, dtype=t.int32, device="cuda"), t.empty(cnt, dtype=t.int32).pin_memory())

    def source_buffer(self):
        return self.torch.empty(2 * GROUP, dtype=self.torch.int32).pin_memory()

    def warm(self, slot, kinds, src: int) -> None:
        """First use of each call on the slot's handle (workspace set-up, graph instantiation)."""
        alb = self.alb
        slot.h_srcs[0] = src
        slot.h_srcs[GROUP] = src
        if "bfs" in kinds:
            alb.alb_bfs_batch(slot.G.h, slot.h_srcs[:1], 1, slot.bufs["bfs"][0], slot.stream)
        if "sssp" in kinds:
            alb.alb_sssp_batch(slot.G.h, slot.h_srcs[GROUP:GROUP + 1], 1, slot.bufs["sssp"][0], slot.stream)
        if "cc" in kinds:
            alb.alb_cc(slot.G.h, slot.bufs["cc"][0], slot.stream)
        slot.stream.synchronize()

    def launch(self, slot, bq, sq, cq):
        """One batch on the slot's stream; returns an event that completes with its copies."""
        t, alb = self.torch, self.alb
        n = slot.n
        # the slot's pinned source list is free: its previous batch has completed
        for j, r in enumerate(bq):
            slot.h_srcs[j] = r.src
        for j, r in enumerate(sq):
            slot.h_srcs[GROUP + j] = r.src
        with t.cuda.stream(slot.stream):
            if bq:
                d, h = slot.bufs["bfs"]
                alb.alb_bfs_batch(slot.G.h, slot.h_srcs[:len(bq)], len(bq), d, slot.stream)
                h[: len(bq) * n].copy_(d[: len(bq) * n], non_blocking=True)
            if sq:
                d, h = slot.bufs["sssp"]
                alb.alb_sssp_batch(slot.G.h, slot.h_srcs[GROUP:GROUP + len(sq)], len(sq), d, slot.stream)
                h[: len(sq) * n].copy_(d[: len(sq) * n], non_blocking=True)
            if cq:
                d, h = slot.bufs["cc"]
                alb.alb_cc(slot.G.h, d, slot.stream)
                h.copy_(d, non_blocking=True)
            ev = t.cuda.Event()
            ev.record(slot.stream)
        return ev

    def done(self, ev) -> bool:
        return ev.query()

    def result(self, slot, kind: str, j: int) -> np.ndarray:
        h = slot.bufs[kind][1]
        n = slot.n
        if kind == "cc":
            return h.numpy().view(np.uint32).copy()
        return h[j * n:(j + 1) * n].numpy().view(np.uint32).copy()

    def check(self, slot) -> None:
        if not self.checked:
            return
        rec = self.alb.alb_debug_check(slot.G.h)
        if rec[0]:
            raise RuntimeError(f"bounds check failed on a graph of n={slot.n}: code {rec[0]} index "
                               f"{rec[1]} bound {rec[2]} count {rec[3]}")

    def synchronize(self) -> None:
        self.torch.cuda.synchronize()

    def release_buffers(self) -> None:
        # freed tensors go back to torch's cache, which Admission counts as free
        pass

    def close(self) -> None:
        t = self.torch
        t.cuda.synchronize()
        if self.parts is not None:
            # the partitions' streams go last, after every buffer the allocator may still
            # associate with them
            import gc
            gc.collect()
            t.cuda.synchronize()
            t.cuda.empty_cache()
            for p in self.parts:
                p.close()
            self.parts = None


class _Slot:
    """One handle (the graph's own, or a clone sharing its CSR) with its stream and buffers.
    Result buffers and the handle's per-kind workspaces are set up on first need."""

    def __init__(self, backend, G, n: int, stream, clone: bool):
        self.backend = backend
        self.G = G
        self.n = n
        self.stream = stream
        self.clone = clone
        self.bufs: dict = {}       # kind -> (device, host) result buffers
        self.warmed: set = set()   # kinds whose first call has run on the handle
        self.h_srcs = backend.source_buffer()
        self.busy = None           # (event, bfs, sssp, cc requests, launch time) while in flight
        self.last_used = 0.0

    def missing_bytes(self, kinds) -> int:
        """Device bytes a batch of `kinds` would still allocate on this slot."""
        need = sum(result_bytes(self.n, k) for k in kinds if k not in self.bufs)
        if any(k in ("bfs", "sssp") for k in kinds) and not (self.warmed & {"bfs", "sssp"}):
            need += BATCH_WS_PER_VERTEX * self.n
        return need

    def ensure(self, kinds, warm_src: int) -> None:
        new = [k for k in kinds if k not in self.warmed]
        for k in kinds:
            if k not in self.bufs:
                self.bufs[k] = self.backend.buffers(self.n, k)
        if new:
            self.backend.warm(self, new, warm_src)
            self.warmed.update(new)

    def release(self) -> int:
        """Drop result buffers and the handle's cached workspaces (idle slot only)."""
        freed = sum(result_bytes(self.n, k) for k in self.bufs)
        self.bufs = {}
        self.warmed = set()
        self.backend.release_buffers()
        freed += self.backend.trim(self.G)
        return freed


class _Graph:
    """A graph of the server: its request queues and, while resident, one or more slots."""

    def __init__(self, server, csr, gid: int, priority: int, big: bool, max_slots: int):
        self.server = server
        self.csr = csr
        self.gid = gid
        self.n = csr.n
        self.m = csr.m
        self.deg = csr.degrees().astype(np.int64)
        self.hot = int(np.argmax(self.deg)) if self.n else 0   # warm-up source
        self.priority = priority
        self.big = big
        self.max_slots = max_slots
        self.part = server.backend.part_for(big)
        self.slots: list[_Slot] = []
        self.queue = {k: deque() for k in KINDS}
        self.log = []          # (seconds in flight, #bfs, #sssp, #cc) per completed batch
        self.last_used = 0.0
        self.uploads = 0

    @property
    def resident(self) -> bool:
        return bool(self.slots)

    def upload_bytes(self) -> int:
        return csr_bytes(self.csr) + ROUND_WS_PER_VERTEX * self.n

    def clone_bytes(self) -> int:
        return ROUND_WS_PER_VERTEX * self.n

    def batch_bytes(self, slot: _Slot, nb: int, ns: int, nc: int) -> int:
        """Device bytes a batch (nb bfs, ns sssp, nc cc queries) needs beyond what its slot holds."""
        kinds = [k for k, c in zip(KINDS, (nb, ns, nc)) if c]
        return slot.missing_bytes(kinds)

    def upload(self) -> None:
        be = self.server.backend
        grid = min(self.server.ctas_per_sm * be.sms(self.part), max(16, -(-self.m // EDGES_PER_CTA)))
        G = be.upload(self.csr, grid, self.hot if self.server.tune and self.uploads == 0 else None)
        self.uploads += 1
        self.slots = [_Slot(be, G, self.n, be.stream(self.priority, self.part), clone=False)]

    def add_slot(self) -> _Slot:
        be = self.server.backend
        s = _Slot(be, be.clone(self.slots[0].G), self.n, be.stream(self.priority, self.part), clone=True)
        self.slots.append(s)
        return s

    def idle(self) -> bool:
        return all(s.busy is None for s in self.slots)

    def queued(self) -> int:
        return sum(len(q) for q in self.queue.values())

    def evict(self) -> None:
        be = self.server.backend
        for s in reversed(self.slots):
            s.bufs = {}
            be.destroy(s.G)
        self.slots = []
        be.release_buffers()

    def close(self):
        if self.slots:
            self.evict()


class Server:
    """Continuous batching over resident graphs; see the module docstring."""

    def __init__(self, graphs, *, tune: bool = True, keep_results: bool = False,
                 hbm_reserve: int = 1 << 30, big_graph_edges: int = 50_000_000, big_slots: int = 2,
                 ctas_per_sm: int = 2, small_sms: int = 0, lazy: bool = False, backend=None,
                 mem_get_info=None):
        self.backend = backend if backend is not None else CudaBackend(small_sms)
        be = self.backend
        self.tune = tune
        self.ctas_per_sm = ctas_per_sm
        # an injected mem_get_info replaces the whole view of free memory (the device's free
        # bytes and the caching allocator's idle blocks)
        self.adm = (Admission(mem_get_info, hbm_reserve) if mem_get_info is not None
                    else Admission(be.mem_get_info, hbm_reserve, be.cached))
        # smaller graphs get higher stream priority, so their short rounds are scheduled
        # between the round kernels of large graphs instead of waiting behind them
        lo, hi = be.priority_range()
        order = np.argsort(np.argsort([g.m for g in graphs]))
        self.graphs = [_Graph(self, g, i, hi if order[i] < len(graphs) // 2 else lo,
                              g.m >= big_graph_edges, big_slots if g.m >= big_graph_edges else 1)
                       for i, g in enumerate(graphs)]
        self.keep = keep_results
        self.results: dict[int, np.ndarray] = {}
        self.batches = 0
        self.deferred = 0     # batch formations postponed for lack of free device memory
        self.evictions = 0    # slots released, workspaces trimmed or graphs evicted for room
        self.admitted_slots = 0  # extra slots created while serving
        self.edges = 0        # traversed-edge units of completed requests (m of the graph each)
        self.admit_log: list[tuple[int, str, int]] = []  # (graph, kind, request id) in launch order
        if not lazy:
            # everything up front (and warmed), while memory allows: nothing is set up while
            # kernels run
            for gr in self.graphs:
                if self.adm.admits(gr.upload_bytes()):
                    gr.upload()
            for gr in self.graphs:
                while gr.resident and len(gr.slots) < gr.max_slots and \
                        self.adm.admits(gr.clone_bytes() + gr.slots[0].missing_bytes(KINDS) * 2):
                    gr.add_slot()
                for s in gr.slots:
                    if self.adm.admits(s.missing_bytes(KINDS)):
                        s.ensure(KINDS, gr.hot)
        slots = sum(max(1, g.max_slots) for g in self.graphs)
        queues = int(os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"))
        if backend is None and slots + 1 > queues:
            import warnings
            warnings.warn(f"{slots} slot streams share {queues} hardware work queues; set "
                          f"CUDA_DEVICE_MAX_CONNECTIONS={min(32, slots + 1)} before CUDA starts")

    @property
    def reserve(self) -> int:
        return self.adm.reserve

    @reserve.setter
    def reserve(self, v: int) -> None:
        self.adm.reserve = int(v)

    def close(self):
        self.backend.synchronize()
        for g in self.graphs:
            g.close()
        self.backend.close()

    # ---------------------------------------------------------------- memory

    def _make_room(self, need: int, keep: _Graph) -> bool:
        """Evict idle resources of graphs other than `keep`, least recently used first, until
        `need` bytes are admitted. Returns whether they are."""
        while not self.adm.admits(need):
            cands = []
            for g in self.graphs:
                if g is keep or not g.resident or not g.idle():
                    continue
                for s in g.slots[1:]:
                    cands.append((0, s.last_used, "slot", g, s))
                for s in g.slots:
                    if s.bufs or s.warmed:
                        cands.append((1, s.last_used, "release", g, s))
                if g.queued() == 0:
                    cands.append((2, g.last_used, "graph", g, None))
            if not cands:
                return False
            _, _, what, g, s = min(cands, key=lambda c: (c[0], c[1]))
            if what == "slot":
                s.bufs = {}
                self.backend.destroy(s.G)
                g.slots.remove(s)
                self.backend.release_buffers()
            elif what == "release":
                s.release()
            else:
                g.evict()
            self.evictions += 1
        return True

    # ------------------------------------------------------------- batches

    def _take(self, gr: _Graph):
        bq = [gr.queue["bfs"].popleft() for _ in range(min(GROUP, len(gr.queue["bfs"])))]
        sq = [gr.queue["sssp"].popleft() for _ in range(min(GROUP, len(gr.queue["sssp"])))]
        cq = list(gr.queue["cc"])
        gr.queue["cc"].clear()
        return bq, sq, cq

    def _put_back(self, gr: _Graph, bq, sq, cq) -> None:
        for q, items in (("bfs", bq), ("sssp", sq), ("cc", cq)):
            gr.queue[q].extendleft(reversed(items))

    def _launch(self, gr: _Graph, s: _Slot, now: float = 0.0) -> bool:
        bq, sq, cq = self._take(gr)
        need = gr.batch_bytes(s, len(bq), len(sq), len(cq))
        if not self.adm.admits(need) and not self._make_room(need, gr):
            # not admitted: back to the front of the queues, retried when memory frees up
            self._put_back(gr, bq, sq, cq)
            self.deferred += 1
            return False
        kinds = [k for k, q in zip(KINDS, (bq, sq, cq)) if q]
        s.ensure(kinds, gr.hot)
        ev = self.backend.launch(s, bq, sq, cq)
        for k, q in zip(KINDS, (bq, sq, cq)):
            self.admit_log += [(gr.gid, k, r.rid) for r in q]
        s.busy = (ev, bq, sq, cq, time.perf_counter())
        s.last_used = gr.last_used = now
        self.batches += 1
        return True

    def _admit_graph(self, gr: _Graph) -> bool:
        need = gr.upload_bytes()
        if not self.adm.admits(need) and not self._make_room(need, gr):
            self.deferred += 1
            return False
        gr.upload()
        return True

    def _maybe_add_slot(self, gr: _Graph) -> None:
        """A large graph whose slots are all busy and that has a full group queued gets another
        slot while memory admits it."""
        if len(gr.slots) >= gr.max_slots or any(s.busy is None for s in gr.slots):
            return
        if max(len(gr.queue["bfs"]), len(gr.queue["sssp"])) < GROUP:
            return
        kinds = [k for k in KINDS if gr.queue[k]]
        probe = _Slot.__new__(_Slot)
        probe.n, probe.bufs, probe.warmed = gr.n, {}, set()
        if self.adm.admits(gr.clone_bytes() + probe.missing_bytes(kinds)):
            gr.add_slot()
            self.admitted_slots += 1

    def _complete(self, gr: _Graph, s: _Slot, now: float):
        ev, bq, sq, cq, t_launch = s.busy
        self.backend.check(s)
        gr.log.append((time.perf_counter() - t_launch, len(bq), len(sq), len(cq)))
        self.edges += gr.m * (len(bq) + len(sq) + len(cq))
        for kind, q in (("bfs", bq), ("sssp", sq), ("cc", cq)):
            for j, r in enumerate(q):
                r.done = now
                if self.keep:
                    self.results[r.rid] = self.backend.result(s, kind, j)
        s.busy = None
        s.last_used = gr.last_used = now

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
                    if s.busy is not None and self.backend.done(s.busy[0]):
                        before = sum(len(x) for x in s.busy[1:4])
                        self._complete(gr, s, time.perf_counter() - t0)
                        pending -= before
                        progressed = True
            for gr in self.graphs:
                if not gr.queued():
                    continue
                if not gr.resident and not self._admit_graph(gr):
                    continue
                self._maybe_add_slot(gr)
                for s in list(gr.slots):
                    if s.busy is None and gr.queued():
                        progressed |= self._launch(gr, s, time.perf_counter() - t0)
            if not progressed:
                time.sleep(0.0001)
        return time.perf_counter() - t0


def one_at_a_time(graphs_or_server, requests: list[Request], *, keep_results: bool = False):
    """Reference path: one request at a time, in arrival order, each with its own call on one
    stream (alb_bfs / alb_sssp / alb_cc), results copied to the host. Returns (seconds, results)."""
    srv = graphs_or_server
    be = srv.backend
    torch, alb = be.torch, be.alb
    res = {}
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        gr = srv.graphs[r.graph]
        if not gr.resident:
            gr.upload()
        s = gr.slots[0]
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
