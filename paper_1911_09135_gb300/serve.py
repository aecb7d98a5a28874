"""Continuous-batching query server over resident graphs (bfs / sssp / cc).

Graphs are uploaded once and stay resident, each with its own CUDA stream (a slot). Requests
arrive open-loop; each is queued on its graph. Whenever a graph's slot is idle and queued work
exists, the server forms one batch from that graph's queue - up to 32 bfs sources and 32 sssp
sources (one multi-source group each, sharing every CSR read: alb_bfs_batch / alb_sssp_batch)
plus every queued cc query (one alb_cc serves them all) - admits it only if free device memory
covers its output buffers, launches it on the slot's stream and copies the requested rows to
pinned host memory. Slots of different graphs run concurrently on the device, and requests that
arrive meanwhile wait for the next batch of their graph. A request's latency runs from its
arrival to the completion of its result's device-to-host copy.

All traversal work runs in libalb.so; this module only schedules calls.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import alb

GROUP = 32
KINDS = ("bfs", "sssp", "cc")


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
    def __init__(self, torch, csr, tune: bool):
        self.torch = torch
        self.n = csr.n
        self.m = csr.m
        self.deg = csr.degrees().astype(np.int64)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
        self.G = alb.Graph(csr.n, dev(csr.offsets), dev(csr.indices), dev(csr.weights),
                           symmetric=csr.symmetric)
        self.stream = torch.cuda.Stream()
        self.queue = {k: deque() for k in KINDS}
        self.busy = None      # (event, batch info) while a batch is in flight
        # pinned host staging for one batch's results
        self.h_bfs = torch.empty(GROUP * csr.n, dtype=torch.int32).pin_memory()
        self.h_sssp = torch.empty(GROUP * csr.n, dtype=torch.int32).pin_memory()
        self.h_cc = torch.empty(csr.n, dtype=torch.int32).pin_memory()
        if tune:
            src = int(np.argmax(self.deg))
            for k in KINDS:
                self.G.autotune(k, src, reps=1)

    def batch_bytes(self, nb, ns, nc) -> int:
        return 4 * self.n * (nb + ns + (1 if nc else 0))

    def close(self):
        self.G.close()


class Server:
    """One slot per resident graph; see the module docstring."""

    def __init__(self, graphs, *, tune: bool = True, keep_results: bool = False,
                 hbm_reserve: int = 1 << 30):
        import torch
        self.torch = torch
        self.slots = [_Slot(torch, g, tune) for g in graphs]
        self.keep = keep_results
        self.reserve = hbm_reserve
        self.results: dict[int, np.ndarray] = {}
        self.batches = 0
        self.deferred = 0     # batch formations postponed for lack of free device memory
        self.edges = 0        # traversed-edge units of completed requests (m of the graph each)

    def close(self):
        for s in self.slots:
            s.close()

    def _free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info()
        cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        return int(free + cached)

    def _launch(self, s: _Slot):
        torch = self.torch
        bq = [s.queue["bfs"].popleft() for _ in range(min(GROUP, len(s.queue["bfs"])))]
        sq = [s.queue["sssp"].popleft() for _ in range(min(GROUP, len(s.queue["sssp"])))]
        cq = list(s.queue["cc"])
        s.queue["cc"].clear()
        need = s.batch_bytes(len(bq), len(sq), len(cq))
        if self._free_bytes() - need < self.reserve:
            # not admitted: back to the front of the queues, retried when memory frees up
            for q, items in (("bfs", bq), ("sssp", sq), ("cc", cq)):
                s.queue[q].extendleft(reversed(items))
            self.deferred += 1
            return False
        n = s.n
        with torch.cuda.stream(s.stream):
            bufs = []
            if bq:
                srcs = torch.tensor([r.src for r in bq], dtype=torch.int32).pin_memory()
                out = torch.empty(len(bq) * n, dtype=torch.int32, device="cuda")
                alb.alb_bfs_batch(s.G.h, srcs, len(bq), out, s.stream)
                s.h_bfs[: len(bq) * n].copy_(out, non_blocking=True)
                bufs += [srcs, out]
            if sq:
                srcs = torch.tensor([r.src for r in sq], dtype=torch.int32).pin_memory()
                out = torch.empty(len(sq) * n, dtype=torch.int32, device="cuda")
                alb.alb_sssp_batch(s.G.h, srcs, len(sq), out, s.stream)
                s.h_sssp[: len(sq) * n].copy_(out, non_blocking=True)
                bufs += [srcs, out]
            if cq:
                out = torch.empty(n, dtype=torch.int32, device="cuda")
                alb.alb_cc(s.G.h, out, s.stream)
                s.h_cc.copy_(out, non_blocking=True)
                bufs.append(out)
            ev = torch.cuda.Event()
            ev.record(s.stream)
        s.busy = (ev, bq, sq, cq, bufs)
        self.batches += 1
        return True

    def _complete(self, s: _Slot, now: float):
        ev, bq, sq, cq, bufs = s.busy
        n = s.n
        self.edges += s.m * (len(bq) + len(sq) + len(cq))
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
        del bufs

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
                self.slots[r.graph].queue[r.kind].append(r)
                i += 1
            progressed = False
            for s in self.slots:
                if s.busy is not None and s.busy[0].query():
                    before = sum(len(x) for x in s.busy[1:4])
                    self._complete(s, time.perf_counter() - t0)
                    pending -= before
                    progressed = True
                if s.busy is None and any(s.queue[k] for k in KINDS):
                    progressed |= self._launch(s)
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
        s = srv.slots[r.graph]
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


def latency_stats(requests: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in requests], dtype=np.float64) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "max_ms": round(float(lat.max()), 3)}
