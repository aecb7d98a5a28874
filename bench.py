#!/usr/bin/env python3
"""Benchmark of the ALB graph-analytics path (arXiv:1911.09135) on GB300.

One step = the whole hot path over one synthetic graph: bfs and sssp from the
highest-degree vertex, cc, PageRank (d = 0.85, tol 1e-6) and k-core (k = 32)
on the severe-imbalance graph (RMAT scale 24, edge factor 16, seed 3, plus 16
hubs of 2^22 uniform targets, symmetrised, weights in [1, 100]); every round of
every app runs through libalb.so. Graph construction and upload are outside the
timed region (as in the paper, Sec. 5); the `e2e` figure puts them back in.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle instead
(on a bounded sample of the same workload) and prints the same line shape.
Multi-GPU runs (torchrun) are independent replicas: the path does not shard.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS per app (BFS/SSSP/CC/PR) on 1 GB300; % HBM peak; batched p50/p99 latency"
UNIT = "GTEPS"
INF = 0xFFFFFFFF
APPS = ("bfs", "sssp", "cc", "pr", "kcore")
KCORE_K = 32
PR_D, PR_TOL, PR_MAX = 0.85, 1e-6, 1000

# algorithmic bytes: per expanded edge and per processed (frontier) vertex
BYTES_PER_EDGE = {"bfs": 8, "sssp": 12, "cc": 8, "kcore": 8, "pr": 8}
BYTES_PER_VERTEX = {"bfs": 16, "sssp": 20, "cc": 20, "kcore": 16, "pr": 20}
KERNEL_NAMES = {
    ("bfs", "twc"): "k_inspect<BfsOp>", ("bfs", "lb"): "k_lb<BfsOp>",
    ("sssp", "twc"): "k_inspect<SsspOp>", ("sssp", "lb"): "k_lb<SsspOp>",
    ("cc", "twc"): "k_inspect<CcOp>", ("cc", "lb"): "k_lb<CcOp>",
    ("kcore", "twc"): "k_inspect<KcoreOp>", ("kcore", "lb"): "k_lb<KcoreOp>",
    ("pr", "twc"): "k_pr_pull", ("pr", "lb"): "k_pr_hub",
}
# the files that define each kernel family's device code (traffic.json is keyed to their hash)
_CSRC = "paper_1911_09135_gb300/csrc/alb/"
KERNEL_SOURCES = {
    "k_pr_": [_CSRC + f for f in ("alb_pagerank.cu", "alb_device.cuh", "alb_internal.cuh")],
    "k_": [_CSRC + f for f in ("alb_kernels.cuh", "alb_device.cuh", "alb_internal.cuh")],
}


UNITS_DESC = ("traversed edges (CSR entries), the same definition for the GPU path and the "
              "oracle: bfs and sssp = degree sum of the reached vertices (Graph500 style); "
              "cc = m (every entry is examined at least once; label propagation's repeat "
              "visits are not counted); kcore = degree sum of the peeled vertices (the entries "
              "peeling examines); pr = m x iterations")


def unit_counts(g, out: dict, pr_iters: int) -> dict:
    """Units of one step of each app from its results (numpy arrays): see UNITS_DESC."""
    deg = g.degrees().astype(np.int64)
    u = {}
    for a, r in out.items():
        if a in ("bfs", "sssp"):
            u[a] = int(deg[np.asarray(r).view(np.uint32) != INF].sum())
        elif a == "cc":
            u[a] = int(g.m)
        elif a == "kcore":
            u[a] = int(deg[np.asarray(r).view(np.uint32) == 0].sum())
        elif a == "pr":
            u[a] = int(g.m) * int(pr_iters)
    return u


def step_config(g, desc, apps, src, world) -> dict:
    """The workload of one step, identical in the GPU arm and the reference (oracle) arm."""
    return {"workload": f"{g.name}: {desc}", "n": g.n, "m": g.m, "apps": list(apps),
            "source": int(src), "kcore_k": KCORE_K, "pagerank": {"d": PR_D, "tol": PR_TOL},
            "l2": l2_note(g),
            "parallelism": f"replicas x{world} (the path does not shard)", "units": UNITS_DESC}


def l2_note(g) -> str:
    csr = 4 * (g.n + 1) + 4 * g.m * (2 if g.weights is not None else 1)
    if csr > (129 << 20):
        return f"no flush: the CSR ({csr / 1e9:.2f} GB) is larger than L2 (129 MB)"
    return f"no flush: the CSR ({csr / 1e6:.1f} MB) fits L2; a launch-bound configuration"


def tune_source(g, src: int) -> int:
    """A vertex other than the timed source for the autotuner's bfs/sssp trials (seeded draw
    among the non-isolated vertices), so the knobs are not fitted to the timed query."""
    cand = np.nonzero(g.degrees() > 0)[0]
    cand = cand[cand != src]
    if cand.size == 0:
        return int(src)
    rng = np.random.Generator(np.random.Philox(key=7))
    return int(cand[rng.integers(0, cand.size)])


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["alb", "reference"], default="alb")
    ap.add_argument("--workload", choices=["rmat24-hubs", "rmat22-hubs", "rmat22", "rmat16",
                                           "batch-sources", "batch-graphs", "ablation", "serve",
                                           "cta-load"],
                    default="rmat24-hubs",
                    help="batch-*: batched vs one-query-at-a-time throughput (separate line)")
    ap.add_argument("--apps", default="", help="comma list restricting the workload's apps")
    ap.add_argument("--exec-mode", choices=["graph", "host"], default="graph",
                    help="graph: device-side round loop (default); host: one launch per kernel "
                         "(ncu cannot profile kernels inside graphs with conditional nodes)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the paper's default threshold rule instead of the autotuned knobs")
    ap.add_argument("--hub-threshold", type=int, default=None,
                    help="a fixed huge-vertex threshold for every app (no autotuning), e.g. for "
                         "the threshold study or a profiling capture")
    ap.add_argument("--batch-threshold", type=int, default=None,
                    help="batch-sources: a fixed threshold for the batched calls instead of the "
                         "search over candidates")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-roofline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--small-sms", type=int, default=0,
                    help="serve: an SM partition of this many SMs for the small graphs (0 = none)")
    ap.add_argument("--big-slots", type=int, default=2, help="serve: slots per large graph")
    ap.add_argument("--batch-scale", type=int, default=22,
                    help="batch-sources: RMAT scale of the graph (22 = the batched configuration; "
                         "smaller scales for profiling captures)")
    return ap.parse_args()


def _gen_threads() -> int:
    """Generator threads for this process: its share of the host's cores when torchrun starts
    several ranks on one node (the output does not depend on the thread count)."""
    local = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
    return max(1, len(os.sched_getaffinity(0)) // max(1, local))


def workload(name):
    from paper_1911_09135_gb300 import graphgen as gg
    nt = _gen_threads()
    if name == "rmat24-hubs":
        g = gg.rmat24_hubs_sym(nthreads=nt)
        desc = ("RMAT(a=.57,b=.19,c=.19) scale 24, edge factor 16, seed 3, + 16 hubs x 2^22 "
                "uniform targets, symmetrised, dedup, weights U[1,100]")
        apps = APPS
    elif name == "rmat22-hubs":
        g = gg.scaled_hub_graph(22, nthreads=nt)
        desc = ("RMAT scale 22, edge factor 16, seed 3, + 16 hubs x 2^20 uniform targets, "
                "symmetrised, dedup, weights U[1,100] (small member of the severe-imbalance family)")
        apps = APPS
    elif name == "rmat22":
        g = gg.rmat22_sym(nthreads=nt)
        desc = "RMAT scale 22, edge factor 16, seed 2, symmetrised, dedup, weights U[1,100]"
        apps = ("bfs", "sssp")
    else:
        g = gg.rmat16_directed(nthreads=nt)
        desc = "RMAT scale 16, edge factor 16, seed 1, directed, dedup"
        apps = ("bfs",)
    return g, desc, apps


# ------------------------------------------------------------------ distributed plumbing

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def done(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class TimedRegion:
    """Barrier + device synchronisation on both sides and nvidia-smi clock samples throughout
    (the clocks record of a bench line)."""

    def __init__(self, dist):
        self.dist = dist
        self.sampler = ClockSampler(dist.local)
        self.clocks = None

    def __enter__(self):
        import torch
        self.dist.barrier()
        torch.cuda.synchronize()
        self.sampler.start()
        return self

    def __exit__(self, *exc):
        import torch
        torch.cuda.synchronize()
        self.dist.barrier()
        self.clocks = self.sampler.stop()
        return False


# ------------------------------------------------------------------ GPU arm

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_src_sha(kernel: str) -> str:
    """Hash of the sources that define `kernel` (by name prefix: PageRank's or the traversals')."""
    files = next(v for k, v in KERNEL_SOURCES.items() if kernel.startswith(k))
    h = hashlib.sha256()
    for rel in files:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, units: float):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if still current."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(kernel)
    if not ent or ent.get("src_sha") != kernel_src_sha(kernel):
        return None
    return ent.get("dram_bytes_per_launch")


class GpuStep:
    def __init__(self, g, apps, alb, torch):
        self.g, self.apps, self.alb, self.torch = g, apps, alb, torch
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
        self.d_off, self.d_idx = dev(g.offsets), dev(g.indices)
        self.d_w = dev(g.weights) if g.weights is not None else None
        self.G = alb.Graph(g.n, self.d_off, self.d_idx, self.d_w, symmetric=g.symmetric)
        self.src = g.max_degree_vertex()
        n = g.n
        self.out = {a: torch.empty(n, dtype=torch.float32 if a == "pr" else torch.int32, device="cuda")
                    for a in apps}
        self.l1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.iters = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run_app(self, a, stream=None):
        alb, G = self.alb, self.G
        if a == "bfs":
            alb.alb_bfs(G.h, self.src, self.out[a], stream)
        elif a == "sssp":
            alb.alb_sssp(G.h, self.src, self.out[a], stream)
        elif a == "cc":
            alb.alb_cc(G.h, self.out[a], stream)
        elif a == "pr":
            alb.alb_pagerank(G.h, PR_D, PR_TOL, PR_MAX, self.out[a], self.l1, self.iters, stream)
        elif a == "kcore":
            alb.alb_kcore(G.h, KCORE_K, self.out[a], stream)

    def calibrate(self):
        """One untimed pass: traversed-edge units and kernel launches per app."""
        g = self.g
        launches, stats, outs = {}, {}, {}
        pr_iters = 0
        for a in self.apps:
            self.run_app(a)
            st = self.G.stats()
            stats[a] = st
            outs[a] = self.out[a].cpu().numpy()
            if a == "pr":
                pr_iters = int(self.iters.item())
            if a == "pr":
                # set-args, init, output; per iteration the pull and the finalize, and with huge
                # vertices the hub kernel, the first-level hub sums and the hub finish
                nh = st["max_hub_count"]
                launches[a] = 3 + st["rounds"] * (2 + (3 if nh else 0))
            else:
                launches[a] = 2 + st["rounds"] + st["hub_rounds"] + (1 if a == "kcore" else 0)
        return unit_counts(g, outs, pr_iters), launches, stats

    def roofline_pass(self):
        """Each app once more in the host-loop mode with every kernel timed by CUDA events."""
        rows = []
        for a in self.apps:
            p0 = self.G.params(a)
            self.G.set_app_params(a, exec_mode=1, profile=1)
            self.run_app(a)
            st = self.G.stats()
            self.G.set_app_params(a, exec_mode=p0.exec_mode, profile=0)
            n_front = st["pushes"] + (self.g.n if a in ("cc", "pr") else 1)
            if a == "pr":
                n_front = self.g.n * st["rounds"]
            for cls, ms, nl, edges in (("twc", st["ms_inspect"], st["n_inspect"], st["edges_twc"]),
                                       ("lb", st["ms_lb"], st["n_lb"], st["edges_lb"])):
                if nl == 0 or ms <= 0:
                    continue
                byts = BYTES_PER_EDGE[a] * edges + (BYTES_PER_VERTEX[a] * n_front if cls == "twc" else 0)
                rows.append({"app": a, "cls": cls, "kernel": KERNEL_NAMES[(a, cls)], "ms": ms,
                             "launches": nl, "bytes": byts, "edges": edges})
        return rows

    def close(self):
        self.G.close()


def gpu_arm(args, dist):
    import torch
    from paper_1911_09135_gb300 import alb

    torch.cuda.set_device(dist.local)
    alb.load()
    g, desc, apps = workload(args.workload)
    if args.apps:
        apps = tuple(a for a in args.apps.split(",") if a in apps)
    step = GpuStep(g, apps, alb, torch)
    if args.hub_threshold is not None:
        args.no_tune = True
        step.G.set_params(hub_threshold=args.hub_threshold)
    # the paper's default rule (threshold = threads of the LB kernel), timed briefly for reference
    paper_rule_ms = None
    if not args.no_tune:
        for a in apps:
            step.run_app(a)
        torch.cuda.synchronize()
        paper_rule_ms = {}
        for a in apps:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(2):
                step.run_app(a)
            e1.record()
            torch.cuda.synchronize()
            paper_rule_ms[a] = round(e0.elapsed_time(e1) / 2, 3)
    # autotuned knobs per app (outside the timed region; results do not depend on them)
    tuned = {}
    tsrc = tune_source(g, step.src)
    if not args.no_tune:
        for a in apps:
            p, _ = step.G.autotune(a, tsrc, reps=2)
            tuned[a] = {"hub_threshold": p.hub_threshold, "twc_cta_min": p.twc_cta_min,
                        "twc_warp_min": p.twc_warp_min, "block_size": p.block_size}
    if args.exec_mode == "host":
        for a in apps:
            step.G.set_app_params(a, exec_mode=1)
    units, launches, cal_stats = step.calibrate()
    units_step = sum(units.values())
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 0)):
        for a in apps:
            step.run_app(a)
    torch.cuda.synchronize()

    clocks = ClockSampler(dist.local)
    ev = {a: [] for a in apps}
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        for a in apps:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step.run_app(a)
            e1.record(stream)
            ev[a].append((e0, e1))
    t1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms_total = t0.elapsed_time(t1)
    ms_max = dist.max(ms_total)
    ms_per_step = ms_max / args.steps
    app_ms = {a: sum(x.elapsed_time(y) for x, y in ev[a]) / args.steps for a in apps}
    step.G.sync()

    total_units = dist.sum(units_step * args.steps)
    value = total_units / (ms_max * 1e-3) / 1e9

    roof = None
    if not args.no_roofline:
        rows = step.roofline_pass()
        if rows:
            top = max(rows, key=lambda r: r["ms"])
            peak, which = measured_peaks()
            achieved = top["bytes"] / (top["ms"] * 1e-3) / 1e9
            traffic = traffic_for(top["kernel"], top["edges"])
            roof = {"bound": "hbm", "kernel": top["kernel"], "achieved": round(achieved, 1),
                    "peak": peak, "peak_source": which, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    # the same launches' measured DRAM bytes (ncu) over their live duration
                    "dram_gbs": (round(traffic / (top["ms"] / top["launches"] * 1e-3) / 1e9, 1)
                                 if traffic else None),
                    "dram_frac": (round(traffic / (top["ms"] / top["launches"] * 1e-3) / 1e9 / peak, 4)
                                  if traffic else None),
                    "algorithmic_bytes_per_launch": int(top["bytes"] / top["launches"]),
                    "avg_launch_ms": round(top["ms"] / top["launches"], 4),
                    "launches": top["launches"],
                    "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
                                for r in sorted(rows, key=lambda r: -r["ms"])]}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_measure(args, g, apps, alb, torch, units_step, dist, tuned)

    # the last timed step's PageRank vector, for its distance to the FP64 oracle (below)
    pr_gpu = step.out["pr"].cpu().numpy().astype(np.float64) if "pr" in apps else None
    step.close()
    pr_oracle = None
    if dist.rank == 0 and pr_gpu is not None:
        # FP64 oracle on the same graph, outside every timed region, on all host cores
        import oracle
        cores = len(os.sched_getaffinity(0))
        t_or = time.perf_counter()
        x_ref, it_ref, _ = oracle.pagerank(g.n, g.offsets, g.indices, PR_D, PR_TOL, PR_MAX,
                                           assume_symmetric=g.symmetric, nthreads=cores,
                                           cache_key=g.key)
        pr_oracle = {"l1_vs_oracle": float(np.abs(pr_gpu - x_ref).sum()), "oracle_iterations": it_ref,
                     "oracle_s": round(time.perf_counter() - t_or, 1), "oracle_cores": cores}
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, apps, step.src, units)

    per_app = {a: {"gteps": round(units[a] / (app_ms[a] * 1e-3) / 1e9, 3),
                   "ms": round(app_ms[a], 3), "units": units[a],
                   "edges_examined": int(cal_stats[a]["edges_twc"] + cal_stats[a]["edges_lb"]),
                   "rounds": cal_stats[a]["rounds"], "hub_rounds": cal_stats[a]["hub_rounds"]}
               for a in apps}
    if "pr" in apps:
        per_app["pr"]["l1_last_change"] = cal_stats["pr"]["pr_l1"]
        if pr_oracle:
            per_app["pr"].update(pr_oracle)
            per_app["pr"]["l1_bound"] = 1e-5
    if paper_rule_ms:
        for a in apps:
            per_app[a]["ms_paper_rule_threshold"] = paper_rule_ms[a]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 (integer apps), f32 (pagerank)", "data": "synthetic",
        "config": step_config(g, desc, apps, step.src, dist.world),
        "run": {"exec_mode": args.exec_mode,
                "knobs": ("autotuned per app by alb_autotune before timing, on a source other "
                          "than the timed one" if tuned
                          else f"fixed threshold {args.hub_threshold}" if args.hub_threshold is not None
                          else "paper's rule: threshold = threads of the LB kernel"),
                "tune_source": int(tsrc) if tuned else None,
                "tuned": tuned or None,
                "hub_threshold": {a: cal_stats[a]["hub_threshold"] for a in apps},
                "lb_threads": cal_stats[apps[0]]["lb_threads"]},
        "per_app": per_app,
        "gpu_launches": int(sum(launches.values()) * args.steps),
        "roofline": roof,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def e2e_measure(args, g, apps, alb, torch, units_step, dist, tuned=None):
    """Same step through the public API with HOST buffers: pinned CSR in, results out."""
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
    h_off, h_idx = pin(g.offsets), pin(g.indices)
    h_w = pin(g.weights) if g.weights is not None else None
    outs = {a: torch.empty(g.n, dtype=torch.float32 if a == "pr" else torch.int32).pin_memory()
            for a in apps}
    h_l1 = torch.zeros(1, dtype=torch.float64).pin_memory()
    h_it = torch.zeros(1, dtype=torch.int32).pin_memory()
    src = g.max_degree_vertex()
    h2d = 4 * (g.n + 1) + 4 * g.m * (2 if h_w is not None else 1)
    d2h = sum(4 * g.n for _ in apps) + (12 if "pr" in apps else 0)

    def one():
        G = alb.Graph(g.n, h_off, h_idx, h_w, symmetric=g.symmetric)
        for a, kw in (tuned or {}).items():
            G.set_app_params(a, **kw)  # the tuned knobs, as a deployed service would keep them
        for a in apps:
            if a == "bfs":
                alb.alb_bfs(G.h, src, outs[a])
            elif a == "sssp":
                alb.alb_sssp(G.h, src, outs[a])
            elif a == "cc":
                alb.alb_cc(G.h, outs[a])
            elif a == "pr":
                alb.alb_pagerank(G.h, PR_D, PR_TOL, PR_MAX, outs[a], h_l1, h_it)
            elif a == "kcore":
                alb.alb_kcore(G.h, KCORE_K, outs[a])
        torch.cuda.synchronize()
        G.close()

    one()  # warm-up (also instantiates the CUDA graphs once)
    dist.barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        one()
    sec = time.perf_counter() - t
    sec = dist.max(sec)
    val = dist.sum(units_step * args.e2e_steps) / sec / 1e9
    return {"value": round(val, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(1e3 * sec / args.e2e_steps, 2),
            "steps": args.e2e_steps,
            "note": "alb.Graph from pinned host CSR + every app with pinned host outputs + destroy"}


# ------------------------------------------------------------------ CPU oracle (baseline)

def oracle_app(g, a, src):
    """One application of the step by the serial CPU oracle, on the full workload graph.
    PageRank runs ONE iteration (its rate per iteration); the others run to completion.
    Returns (result or None, units processed, seconds)."""
    import oracle
    t0 = time.perf_counter()
    if a == "bfs":
        r = oracle.bfs(g.n, g.offsets, g.indices, src)
    elif a == "sssp":
        r = oracle.sssp(g.n, g.offsets, g.indices, g.weights, src)
    elif a == "cc":
        r = oracle.cc(g.n, g.offsets, g.indices)
    elif a == "kcore":
        r = oracle.kcore(g.n, g.offsets, g.indices, KCORE_K)
    else:
        oracle.pagerank(g.n, g.offsets, g.indices, PR_D, PR_TOL, 1, assume_symmetric=g.symmetric,
                        nthreads=1)
        return None, int(g.m), time.perf_counter() - t0
    sec = time.perf_counter() - t0
    return r, unit_counts(g, {a: r}, 0)[a], sec


def mix_rate(step_units: dict, samples: dict) -> float:
    """Throughput (units/s) of the oracle on one step's unit mix: each app's time is its
    measured rate applied to that app's units in the step (PageRank: per-iteration rate times
    the step's iterations). samples[a] = list of (units, seconds)."""
    t = 0.0
    for a, u in step_units.items():
        su = sum(x for x, _ in samples[a])
        ss = sum(y for _, y in samples[a])
        t += u * ss / su if su else 0.0
    return sum(step_units.values()) / t


def cpu_baseline(g, apps, src, step_units):
    """Every app of the step once by the serial oracle (PageRank: one iteration), weighted by the
    GPU step's unit mix."""
    samples = {a: [oracle_app(g, a, src)[1:]] for a in apps}
    sec = sum(s for v in samples.values() for _, s in v)
    return {"value": round(mix_rate(step_units, samples) / 1e9, 4), "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": (f"{' + '.join(a if a != 'pr' else 'pr (1 iteration)' for a in apps)} once each "
                       f"on the full workload graph by the serial CPU oracle ({sec:.1f} s), "
                       f"weighted by the step's units per app; host has "
                       f"{len(os.sched_getaffinity(0))} cores")}


def reference_arm(args, dist):
    """The CPU oracle as it stands on the GPU arm's workload, config, metric and units. A step
    is one application of the five-app mix in turn (bfs, sssp, cc, pr, kcore; PageRank as one
    iteration), run to completion on the full graph; the value is the oracle's throughput on the
    whole step's unit mix (each app's measured rate applied to its units in the step; PageRank's
    iterations are the oracle's own count at tol 1e-6, found once before timing on all cores)."""
    if dist.rank != 0:
        return
    g, desc, apps = workload(args.workload)
    src = g.max_degree_vertex()
    import oracle
    # untimed: PageRank's iteration count at the step's tolerance (the other apps' units come
    # from their first timed result)
    step_units = {}
    pr_iters = 0
    if "pr" in apps:
        _, pr_iters, _ = oracle.pagerank(g.n, g.offsets, g.indices, PR_D, PR_TOL, PR_MAX,
                                         assume_symmetric=g.symmetric,
                                         nthreads=len(os.sched_getaffinity(0)), cache_key=g.key)
        step_units["pr"] = int(g.m) * pr_iters
    cheap = min(apps, key=lambda a: {"kcore": 0, "bfs": 1, "cc": 2, "pr": 3, "sssp": 4}[a])
    for _ in range(max(args.warmup, 0)):
        oracle_app(g, cheap, src)
    order = list(apps)
    plan = [order[i % len(order)] for i in range(max(args.steps, len(order)))]
    samples = {a: [] for a in apps}
    tot_s = 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        for i in range(k, len(plan), args.steps):  # every app at least once over the K steps
            r, u, sec = oracle_app(g, plan[i], src)
            samples[plan[i]].append((u, sec))
            if plan[i] not in step_units:
                step_units[plan[i]] = u
        tot_s += time.perf_counter() - t0
    step_units = {a: step_units[a] for a in apps}
    value = mix_rate(step_units, samples) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_s / args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 (integer apps), f64 (pagerank)", "data": "synthetic", "impl": "reference",
        "config": step_config(g, desc, apps, src, dist.world),
        "per_app": {a: {"units": step_units[a], "samples": len(samples[a]),
                        "gteps": round(sum(x for x, _ in samples[a]) / sum(y for _, y in samples[a]) / 1e9, 4)}
                    for a in apps},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": ("each step: the next app of the five-app mix (PageRank as one "
                                    "iteration) by the serial CPU oracle on the full workload graph"
                                    + (f"; pagerank iterations {pr_iters} (the oracle's own count)"
                                       if "pr" in apps else ""))},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_arm(args, dist):
    """Batched traversal throughput against the one-query-at-a-time plain path, same GPU.

    batch-sources: 128 uniform random sources (seed 4) on rmat22-sym; plain = 128 alb_bfs /
    alb_sssp calls, batched = one alb_bfs_batch / alb_sssp_batch call (groups of 32 sources).
    batch-graphs: 512 RMAT graphs with samples log-uniform in [2^10, 2^22] (seed 4), source 0
    of each; plain = one resident handle per graph, 512 calls; batched = one traversal of their
    disjoint union from all 512 sources (alb_bfs_multi / alb_sssp_multi).
    Outputs stay on the device in both paths; the graphs are resident before timing.
    """
    import torch
    from paper_1911_09135_gb300 import alb, graphgen as gg

    torch.cuda.set_device(dist.local)
    alb.load()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    host_loop = args.exec_mode == "host"
    region = TimedRegion(dist)
    region.__enter__()
    if args.workload == "batch-sources":
        g = (gg.rmat22_sym() if args.batch_scale == 22 else
             gg.rmat(args.batch_scale, 16 << args.batch_scale, 2, symmetrize=True, weighted=True))
        rng = np.random.Generator(np.random.Philox(key=4))
        srcs = rng.integers(0, g.n, size=128).astype(np.uint32)
        d_srcs = dev(srcs)
        # the knobs are chosen on other queries than the timed ones (seed 40)
        tsrcs = np.random.Generator(np.random.Philox(key=40)).integers(0, g.n, size=128).astype(np.uint32)
        d_tsrcs = dev(tsrcs)
        G = alb.Graph(g.n, dev(g.offsets), dev(g.indices), dev(g.weights), symmetric=True)
        out = torch.empty(128 * g.n, dtype=torch.int32, device="cuda")
        n = g.n
        for app, single, batch in (("bfs", alb.alb_bfs, alb.alb_bfs_batch),
                                   ("sssp", alb.alb_sssp, alb.alb_sssp_batch)):
            if args.apps and app not in args.apps.split(","):
                continue
            tuned, _ = G.autotune(app, tune_source(g, int(srcs[0])), reps=2)  # the plain path's knobs
            if host_loop:  # one launch per kernel (profiling captures)
                G.set_app_params(app, exec_mode=1)
            def plain():
                for i, s in enumerate(srcs.tolist()):
                    single(G.h, s, out[i * n:(i + 1) * n])
            ms_plain = timed(plain, max(1, args.steps // 2))
            # the batched path gets its own knobs (multi-source rounds relax every active source
            # of an edge, so the best split between TWC and the LB kernel, the CTA size and the
            # TWC cut-offs can differ), chosen one after another by timing a batch of 128 other
            # sources: the threshold, then the CTA size, then the cut-offs
            def trial_of(**kw):
                G.set_app_params(app, **kw)
                return timed(lambda: batch(G.h, d_tsrcs, 128, out), 1)
            if args.batch_threshold is not None:
                t_best = args.batch_threshold
                G.set_app_params(app, hub_threshold=t_best)
                bknobs = {"block_size": tuned.block_size, "twc_cta_min": tuned.twc_cta_min,
                          "twc_warp_min": tuned.twc_warp_min}
            else:
                cand = sorted({int(tuned.hub_threshold), -1, 1 << 12, 1 << 14, 1 << 16, 1 << 18})
                trial = {t: trial_of(hub_threshold=t) for t in cand}
                t_best = min(trial, key=trial.get)
                G.set_app_params(app, hub_threshold=t_best)
                best = trial[t_best]
                bknobs = {"block_size": tuned.block_size, "twc_cta_min": tuned.twc_cta_min,
                          "twc_warp_min": tuned.twc_warp_min}
                for b in (128, 256, 512):
                    if b == bknobs["block_size"]:
                        continue
                    ms = trial_of(block_size=b)
                    if ms < best:
                        best, bknobs["block_size"] = ms, b
                G.set_app_params(app, block_size=bknobs["block_size"])
                for cm, wm in ((128, 16), (256, 32), (512, 64), (1024, 64), (2048, 128)):
                    if (cm, wm) == (bknobs["twc_cta_min"], bknobs["twc_warp_min"]):
                        continue
                    ms = trial_of(twc_cta_min=cm, twc_warp_min=wm)
                    if ms < best:
                        best, bknobs["twc_cta_min"], bknobs["twc_warp_min"] = ms, cm, wm
                G.set_app_params(app, hub_threshold=t_best, **bknobs)
            ms_batch = timed(lambda: batch(G.h, d_srcs, 128, out), args.steps)
            res[app] = {"queries": 128, "ms_plain": round(ms_plain, 3), "ms_batched": round(ms_batch, 3),
                        "speedup": round(ms_plain / ms_batch, 2),
                        "autotuned": {"hub_threshold": tuned.hub_threshold, "twc_cta_min": tuned.twc_cta_min,
                                      "twc_warp_min": tuned.twc_warp_min, "block_size": tuned.block_size},
                        "batched_hub_threshold": t_best, "batched_knobs": bknobs,
                        "queries_per_s_batched": round(128 / (ms_batch * 1e-3), 1)}
        # rounds of the last group of the timed batch (sssp), for the round-overhead estimate below
        rounds_group = G.stats()["rounds"] if "sssp" in res else None
        G.close()
        # the per-round floor of the CUDA-graph round loop: bfs along a directed path of 4096
        # vertices runs 4096 rounds of one vertex each (a persistent multi-round kernel would
        # replace exactly this cost)
        P = gg.from_edges(4096, [(i, i + 1) for i in range(4095)], None, symmetrize=False, name="path4096")
        GP = alb.Graph(P.n, dev(P.offsets), dev(P.indices))
        po = torch.empty(P.n, dtype=torch.int32, device="cuda")
        ms_path = timed(lambda: alb.alb_bfs(GP.h, 0, po), 3)
        GP.close()
        res["round_floor"] = {"us_per_round": round(1e3 * ms_path / 4096, 2),
                              "rounds_per_sssp_group": rounds_group,
                              "note": "bfs on a 4096-vertex directed path / 4096 rounds"}
        desc = (f"128 sources (seed 4) on rmat{args.batch_scale}-sym (scale {args.batch_scale}, ef 16, "
                f"seed 2, w in [1,100])" + (", host-loop execution" if host_loop else ""))
    else:
        parts = gg.small_graphs(512, seed=4)
        u, base = gg.disjoint_union(parts)
        srcs = base[:-1].astype(np.uint32)
        d_srcs = dev(srcs)
        U = alb.Graph(u.n, dev(u.offsets), dev(u.indices), dev(u.weights), symmetric=True)
        Gs = [alb.Graph(p.n, dev(p.offsets), dev(p.indices), dev(p.weights), symmetric=True)
              for p in parts]
        outs = [torch.empty(p.n, dtype=torch.int32, device="cuda") for p in parts]
        out = torch.empty(u.n, dtype=torch.int32, device="cuda")
        for app, single, multi in (("bfs", alb.alb_bfs, alb.alb_bfs_multi),
                                   ("sssp", alb.alb_sssp, alb.alb_sssp_multi)):
            def plain():
                for G, o in zip(Gs, outs):
                    single(G.h, 0, o)
            ms_plain = timed(plain, max(1, args.steps // 2))
            ms_batch = timed(lambda: multi(U.h, d_srcs, len(parts), out), args.steps)
            res[app] = {"queries": len(parts), "ms_plain": round(ms_plain, 3),
                        "ms_batched": round(ms_batch, 3), "speedup": round(ms_plain / ms_batch, 2),
                        "queries_per_s_batched": round(len(parts) / (ms_batch * 1e-3), 1)}
        for G in Gs:
            G.close()
        U.close()
        desc = (f"512 RMAT graphs, samples log-uniform in [2^10, 2^22] (seed 4), symmetrised, "
                f"w in [1,100]; union n={u.n} m={u.m}; source 0 of each")
    region.__exit__(None, None, None)
    floor = res.pop("round_floor", None)
    q = sum(r["queries"] for r in res.values())
    t = sum(r["ms_batched"] for r in res.values())
    tp = sum(r["ms_plain"] for r in res.values())
    line = {"metric": "batched throughput vs one-query-at-a-time plain path (bfs + sssp)",
            "value": round(q / (t * 1e-3), 1), "unit": "queries/s", "n_gpus": dist.world,
            "steps": args.steps, "warmup": 1, "ms_per_step": round(t, 3),
            "step": "one batched call per app (bfs, then sssp) over all the queries",
            "higher_is_better": True, "speedup_vs_plain": round(tp / t, 2),
            "clocks": region.clocks,
            "config": {"workload": args.workload + ": " + desc}, "per_app": res,
            "round_floor": floor}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def ablation_arm(args, dist):
    """The paper's load-balancing comparison (Sec. 5.1, Table 2; Fig. 5; the threshold study)
    on the severe-imbalance graph: per-app device time under
      alb        - default ALB: threshold = LB threads, cyclic distribution
      alb-blocked- ALB with the blocked distribution (Sec. 4.1)
      twc        - threshold above the maximum degree: TWC only, the LB kernel never runs
      lb-all     - threshold 0: every active vertex goes to the LB kernel (LB for all)
      t=2^k      - the threshold sweep."""
    import torch
    from paper_1911_09135_gb300 import alb

    torch.cuda.set_device(dist.local)
    alb.load()
    g, desc, apps = workload("rmat24-hubs")
    step = GpuStep(g, apps, alb, torch)
    stream = torch.cuda.current_stream()
    settings = [("alb", {}), ("alb-blocked", {"distribution": 1}), ("twc", {"hub_threshold": 1 << 40}),
                ("lb-all", {"hub_threshold": 0})]
    settings += [(f"t=2^{k}", {"hub_threshold": 1 << k}) for k in (8, 10, 12, 14, 16, 18, 20)]
    base = step.G.params()
    table = {}
    region = TimedRegion(dist)
    region.__enter__()
    for name, kw in settings:
        step.G.set_params(**{**{"hub_threshold": base.hub_threshold, "distribution": 0}, **kw})
        row = {}
        for a in apps:
            step.run_app(a)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step.run_app(a)
            e1.record(stream)
            torch.cuda.synchronize()
            st = step.G.stats()
            row[a] = {"ms": round(e0.elapsed_time(e1) / args.steps, 3), "lb_rounds": st["hub_rounds"]}
        table[name] = row
    region.__exit__(None, None, None)
    step.close()
    ms_all = sum(r["ms"] for row in table.values() for r in row.values())
    line = {"metric": "per-app device time (ms) by load-balancing policy", "unit": "ms",
            "higher_is_better": False, "n_gpus": dist.world, "steps": args.steps, "warmup": 1,
            "ms_per_step": round(ms_all, 3),
            "step": "one call of every app under every policy", "clocks": region.clocks,
            "config": {"workload": f"{g.name}: {desc}",
                       "default_threshold": "threads of the LB kernel (alb_params.hub_threshold = -1)"},
            "table": table}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def serve_arm(args, dist):
    """Continuous-batching server over 8 resident graphs (RMAT scales 14, 15, 17, 18, 20, 21,
    23, 24; seeds 500 + i; symmetrised; w in [1,100]); 20,000 bfs/sssp/cc requests with Poisson
    arrivals at 2,000 per second (seed 5), graph and kind uniform. Reports p50/p99 latency,
    throughput and GTEPS (m of the queried graph per request), then the saturation throughput of
    the batched server against one request at a time on the same 4,000 requests."""
    import torch
    from paper_1911_09135_gb300 import alb, graphgen as gg, serve

    torch.cuda.set_device(dist.local)
    alb.load()
    scales = (14, 15, 17, 18, 20, 21, 23, 24)
    graphs = [gg.rmat(sc, 16 << sc, 500 + i, symmetrize=True, weighted=True) for i, sc in enumerate(scales)]
    srv = serve.Server(graphs, tune=True, small_sms=args.small_sms, big_slots=args.big_slots)
    reqs = serve.poisson_requests(graphs, 20000, rate=2000.0, seed=5)
    # warm every slot's cached graphs once
    warm = [serve.Request(-1 - 3 * i - j, 0.0, i, k, int(np.argmax(graphs[i].degrees())))
            for i in range(len(graphs)) for j, k in enumerate(serve.KINDS)]
    srv.run(warm, realtime=False)
    e0 = srv.edges
    region = TimedRegion(dist)
    with region:
        wall = srv.run(reqs, realtime=True, timeout=900)
    lat = serve.latency_stats(reqs)
    per_graph = serve.slot_stats(srv, reqs)
    gteps = (srv.edges - e0) / wall / 1e9
    # the same mix at half the rate, where the server keeps up (latency without queue growth)
    half = serve.poisson_requests(graphs, 10000, rate=1000.0, seed=5)
    for gr in srv.graphs:
        gr.log.clear()  # per-graph batch records of this run only
    e1 = srv.edges
    wall_h = srv.run(half, realtime=True, timeout=900)
    below = {"offered_rate": 1000.0, "requests": len(half), "value": round(len(half) / wall_h, 1),
             "latency": serve.latency_stats(half), "gteps": round((srv.edges - e1) / wall_h / 1e9, 3),
             "batch_ms_mean": [x["batch_ms_mean"] for x in serve.slot_stats(srv, half)]}
    sat = [serve.Request(r.rid, 0.0, r.graph, r.kind, r.src) for r in reqs[:4000]]
    b0 = srv.batches
    t_batched = srv.run(sat, realtime=False, timeout=900)
    nb = srv.batches - b0
    t_plain, _ = serve.one_at_a_time(srv, sat)
    srv.close()
    line = {"metric": "served bfs/sssp/cc requests: p50/p99 latency and throughput", "unit": "queries/s",
            "value": round(len(reqs) / wall, 1), "higher_is_better": True, "n_gpus": dist.world,
            "steps": 1, "warmup": 1, "ms_per_step": round(wall * 1e3, 1),
            "step": "the whole open-loop run of the Poisson requests", "clocks": region.clocks,
            "latency": lat, "gteps": round(gteps, 3), "offered_rate": 2000.0, "requests": len(reqs),
            "wall_s": round(wall, 3), "deferred_admissions": srv.deferred,
            "evictions": srv.evictions, "slots_admitted_while_serving": srv.admitted_slots,
            "per_graph": per_graph,
            "below_saturation": below,
            "saturation": {"requests": len(sat), "batched_s": round(t_batched, 3), "batches": nb,
                           "one_at_a_time_s": round(t_plain, 3),
                           "speedup": round(t_plain / t_batched, 2)},
            "config": {"workload": "8 resident RMAT graphs, scales 14-24 (14,15,17,18,20,21,23,24), "
                                   "seeds 500+i, symmetrised, w in [1,100]; Poisson 2000/s, seed 5",
                       "hardware_queues": int(os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8")),
                       "small_sms": args.small_sms, "big_slots": args.big_slots,
                       "graphs_m": [g.m for g in graphs], "knobs": "autotuned per graph and app"}}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def cta_load_arm(args, dist):
    """Thread-block (CTA) load distribution, the measure of the paper's Figs. 1 and 4: edges
    expanded by each CTA of the TWC part and of the LB kernel, summed over one call, for bfs, sssp
    and pr on the severe-imbalance graph under TWC only (threshold above the maximum degree) and
    ALB (the paper's rule). Reports max / mean / min per kernel and the max-over-mean imbalance."""
    import torch
    from paper_1911_09135_gb300 import alb

    torch.cuda.set_device(dist.local)
    alb.load()
    g, desc, apps = workload("rmat24-hubs")
    step = GpuStep(g, ("bfs", "sssp", "pr"), alb, torch)

    def summary(x):
        x = np.asarray(x, dtype=np.float64)
        if x.size == 0 or x.sum() == 0:
            return None
        return {"ctas": int(x.size), "max": int(x.max()), "mean": round(float(x.mean()), 1),
                "min": int(x.min()), "max_over_mean": round(float(x.max() / x.mean()), 3),
                "p99_over_p50": round(float(np.percentile(x, 99) / max(np.percentile(x, 50), 1)), 3)}

    table = {}
    for policy, t in (("twc", 1 << 40), ("alb", -1)):
        step.G.set_params(hub_threshold=t, cta_stats=1)
        for a in step.apps:
            step.run_app(a)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step.run_app(a)
            e1.record()
            torch.cuda.synchronize()
            twc, lb = step.G.cta_loads()
            table[f"{policy}/{a}"] = {"ms": round(e0.elapsed_time(e1), 3), "twc_kernel": summary(twc),
                                      "lb_kernel": summary(lb)}
    step.close()
    line = {"metric": "per-CTA edges expanded in one call (thread-block load distribution)",
            "unit": "edges", "n_gpus": dist.world, "config": {"workload": f"{g.name}: {desc}"},
            "table": table}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.workload == "serve":
        # one hardware work queue per slot stream: with the default 8, several slots share a FIFO
        # queue and a small graph's batch waits behind a large graph's (set before CUDA starts)
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    dist = Dist()
    if args.workload == "cta-load":
        import torch
        dist.init("nccl" if torch.cuda.is_available() else "gloo")
        try:
            cta_load_arm(args, dist)
        finally:
            dist.done()
        return
    if args.workload == "serve":
        import torch
        dist.init("nccl" if torch.cuda.is_available() else "gloo")
        try:
            serve_arm(args, dist)
        finally:
            dist.done()
        return
    if args.workload == "ablation":
        import torch
        dist.init("nccl" if torch.cuda.is_available() else "gloo")
        try:
            ablation_arm(args, dist)
        finally:
            dist.done()
        return
    if args.workload.startswith("batch-"):
        import torch
        dist.init("nccl" if torch.cuda.is_available() else "gloo")
        try:
            batch_arm(args, dist)
        finally:
            dist.done()
        return
    if args.impl == "reference":
        if dist.world > 1 and dist.rank != 0:
            return
        reference_arm(args, dist)
        return
    import torch
    if dist.world > 1:
        torch.cuda.set_device(dist.local)
    dist.init("nccl" if torch.cuda.is_available() else "gloo")
    try:
        gpu_arm(args, dist)
    finally:
        dist.done()


if __name__ == "__main__":
    main()
