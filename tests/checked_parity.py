"""Parity run of the bounds-checked library (libalb_checked.so), meant for a child process.

Run as ``ALB_CHECKED=1 python -m tests.checked_parity``: every application, the batched and
multi-source calls and the allocation-free BFS run on small graphs under several load-balancing
settings, each result is compared with the CPU oracle, and the checked build's record of
skipped out-of-range accesses (alb_debug_check) must stay all zero on every handle. The
allocation-free BFS reports such a record as ALB_ERR_DEVICE, so its plain success is the check.
Prints ``CHECKED PARITY OK`` at the end; any mismatch raises.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1911_09135_gb300 import graphgen as gg  # noqa: E402
from tests import graphs  # noqa: E402

SETTINGS = [
    dict(hub_threshold=-1),
    dict(hub_threshold=0),
    dict(hub_threshold=3, twc_warp_min=1, twc_cta_min=2),
    dict(hub_threshold=8, twc_warp_min=2, twc_cta_min=4, distribution=1),
    dict(hub_threshold=2, exec_mode=1),
    dict(hub_threshold=4, grid_blocks=3),
]


def main() -> None:
    assert os.environ.get("ALB_CHECKED") == "1", "run with ALB_CHECKED=1"
    import torch

    from paper_1911_09135_gb300 import alb

    alb.load()
    assert alb.alb_checked_build() == 1, "libalb_checked.so was not loaded"
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()
    host = lambda t: t.cpu().numpy().view(np.uint32)

    def make(g):
        return alb.Graph(g.n, dev(g.offsets), dev(g.indices),
                         dev(g.weights) if g.weights is not None else None, symmetric=g.symmetric)

    def clean(G, what):
        rec = alb.alb_debug_check(G.h)
        assert rec == [0, 0, 0, 0], f"{what}: bounds record {rec}"

    hubby = gg.rmat(12, 16 << 12, 7, symmetrize=True, weighted=True, n_hubs=2, hub_degree=1500)
    cases = graphs.all_small() + [graphs.directed_cycle_tail(), hubby]
    checks = 0
    for g in cases:
        src = g.max_degree_vertex() if g.n > 1 else 0
        ref = {"bfs": oracle.bfs(g.n, g.offsets, g.indices, src)}
        if g.weights is not None:
            ref["sssp"] = oracle.sssp(g.n, g.offsets, g.indices, g.weights, src)
        if g.symmetric:
            ref["cc"] = oracle.cc(g.n, g.offsets, g.indices)
            ref["kcore"] = oracle.kcore(g.n, g.offsets, g.indices, 3)
        pr_ref = None
        if g.symmetric:
            pr_ref, _, _ = oracle.pagerank(g.n, g.offsets, g.indices, 0.85, 1e-6, 1000,
                                           assume_symmetric=True)
        for setting in SETTINGS:
            G = make(g)
            G.set_params(**setting)
            o = torch.empty(g.n, dtype=torch.int32, device="cuda")
            for app in ref:
                if app == "bfs":
                    G.bfs(src, o)
                elif app == "sssp":
                    G.sssp(src, o)
                elif app == "cc":
                    G.cc(o)
                else:
                    G.kcore(3, o)
                G.sync()
                assert np.array_equal(host(o), ref[app]), (g.name, setting, app)
                clean(G, f"{g.name} {setting} {app}")
                checks += 1
            if pr_ref is not None:
                r = torch.empty(g.n, dtype=torch.float32, device="cuda")
                G.pagerank(0.85, 1e-6, 1000, r)
                err = float(np.abs(r.cpu().numpy().astype(np.float64) - pr_ref).sum())
                assert err <= 1e-5, (g.name, setting, "pagerank", err)
                clean(G, f"{g.name} {setting} pagerank")
                checks += 1
            G.close()

    # many sources on one graph (groups of 32 on the handle and its worker clones)
    g = hubby
    rng = np.random.Generator(np.random.Philox(key=44))
    srcs = rng.integers(0, g.n, size=40).astype(np.uint32)
    with make(g) as G:
        G.set_params(hub_threshold=512)
        out = torch.empty(40 * g.n, dtype=torch.int32, device="cuda")
        G.bfs_batch(dev(srcs), out)
        G.sync()
        lv = host(out).reshape(40, g.n).copy()
        G.sssp_batch(dev(srcs), out)
        G.sync()
        ds = host(out).reshape(40, g.n).copy()
        clean(G, "batch")
        for i, s in enumerate(srcs.tolist()):
            assert np.array_equal(lv[i], oracle.bfs(g.n, g.offsets, g.indices, s)), ("bfs_batch", i)
            assert np.array_equal(ds[i], oracle.sssp(g.n, g.offsets, g.indices, g.weights, s)), ("sssp_batch", i)
            checks += 2

    # many small graphs as one disjoint union
    parts = [gg.rmat(sc, 16 << sc, 900 + i, symmetrize=True, weighted=True)
             for i, sc in enumerate((4, 6, 9, 5, 11, 7, 4, 10, 8, 6, 12, 5))]
    u, base = gg.disjoint_union(parts)
    with make(u) as U:
        o = torch.empty(u.n, dtype=torch.int32, device="cuda")
        U.bfs_multi(base[:-1].astype(np.uint32), o)
        U.sync()
        lv = host(o).copy()
        U.sssp_multi(base[:-1].astype(np.uint32), o)
        U.sync()
        ds = host(o).copy()
        clean(U, "multi")
    for i, p in enumerate(parts):
        sl = slice(int(base[i]), int(base[i + 1]))
        assert np.array_equal(lv[sl], oracle.bfs(p.n, p.offsets, p.indices, 0)), ("bfs_multi", i)
        assert np.array_equal(ds[sl], oracle.sssp(p.n, p.offsets, p.indices, p.weights, 0)), ("sssp_multi", i)
        checks += 2

    # the allocation-free BFS: a skipped access would be returned as ALB_ERR_DEVICE
    for g, s in ((hubby, hubby.max_degree_vertex()), (gg.rmat16_directed(), 0)):
        o = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for _ in range(2):
            alb.alb_bfs_noalloc(g.n, g.m, dev(g.offsets), dev(g.indices), s, o)
            torch.cuda.synchronize()
            assert np.array_equal(host(o), oracle.bfs(g.n, g.offsets, g.indices, s)), ("noalloc", g.name)
            checks += 1
    torch.cuda.synchronize()
    print(f"CHECKED PARITY OK: {checks} results equal to the oracle, bounds records all zero")


if __name__ == "__main__":
    main()
