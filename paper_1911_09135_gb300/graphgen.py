"""Seeded synthetic graph inputs (shared by the CUDA path's tests/bench and the oracle).

This module draws graphs; it holds none of the traversal arithmetic. Graphs are
returned as host numpy CSR arrays (``uint32`` offsets, indices and optional
weights). The generator itself is native (``csrc/gen/graphgen.cpp``) because a
scale-24 RMAT graph has ~0.6 G entries.

Workload recipes (the paper evaluates on RMAT graphs rmat25-27 and real
power-law graphs, Sec. 5, Table 1; these synthetic graphs of the same RMAT
family and edge factor 16 stand in for them):

* ``rmat16_directed``   - scale 16, edge factor 16, seed 1, directed, BFS from 0.
* ``rmat22_sym``        - scale 22, edge factor 16, seed 2, symmetrised, weights 1..100.
* ``rmat24_hubs_sym``   - scale 24, edge factor 16, seed 3, plus 16 injected hubs with
                          2^22 distinct uniform targets each, symmetrised, weights 1..100.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import json
import math
import os

import numpy as np

from . import _build

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


class _Params(ctypes.Structure):
    _fields_ = [
        ("scale", ctypes.c_uint32),
        ("symmetrize", ctypes.c_uint32),
        ("nsamples", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
        ("a", ctypes.c_double),
        ("b", ctypes.c_double),
        ("c", ctypes.c_double),
        ("n_hubs", ctypes.c_uint32),
        ("hub_degree", ctypes.c_uint32),
        ("weighted", ctypes.c_uint32),
        ("wmin", ctypes.c_uint32),
        ("wmax", ctypes.c_uint32),
        ("nthreads", ctypes.c_int32),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = os.path.join(_build.LIB_DIR, "libalbgen.so")
        if not os.path.exists(path):
            path = _build.build_graphgen()
        lib = ctypes.CDLL(path)
        lib.gg_rmat.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_void_p)]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_n.argtypes = [ctypes.c_void_p]
        lib.gg_n.restype = ctypes.c_uint32
        lib.gg_m.argtypes = [ctypes.c_void_p]
        lib.gg_m.restype = ctypes.c_uint64
        lib.gg_num_hubs.argtypes = [ctypes.c_void_p]
        lib.gg_num_hubs.restype = ctypes.c_uint32
        lib.gg_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4
        lib.gg_copy.restype = ctypes.c_int
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_free.restype = None
        lib.gg_edge_weight.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32]
        lib.gg_edge_weight.restype = ctypes.c_uint32
        _lib = lib
    return _lib


@dataclasses.dataclass
class CSR:
    """Host CSR graph: row ``u`` holds the out-neighbours ``indices[offsets[u]:offsets[u+1]]``."""

    n: int
    offsets: np.ndarray              # uint32[n+1]
    indices: np.ndarray              # uint32[m]
    weights: np.ndarray | None = None  # uint32[m] or None
    symmetric: bool = False
    hubs: np.ndarray | None = None   # injected hub ids, if any
    name: str = ""
    key: str | None = None           # generator graphs: a digest of the recipe and the generator

    @property
    def m(self) -> int:
        return int(self.indices.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64)).astype(np.uint32)

    def max_degree_vertex(self) -> int:
        """Highest out-degree vertex, ties to the smallest id."""
        d = self.degrees()
        return int(np.argmax(d)) if self.n else 0


# On-disk cache of generated graphs: set ALB_GRAPH_CACHE to a directory and every rmat() graph is
# stored there once (numpy .npz) under a digest of its recipe and of the generator's source, and
# loaded from there afterwards (a scale-24 graph takes far longer to draw than to read).
CACHE_ENV = "ALB_GRAPH_CACHE"


def _recipe_key(**recipe) -> str:
    src = os.path.join(_build.CSRC, "gen", "graphgen.cpp")
    h = hashlib.sha256(open(src, "rb").read())
    h.update(json.dumps(recipe, sort_keys=True).encode())
    return h.hexdigest()[:32]


def _cache_load(key: str, name: str, symmetrize: bool) -> CSR | None:
    cdir = os.environ.get(CACHE_ENV)
    path = os.path.join(cdir, key + ".npz") if cdir else None
    if not path or not os.path.exists(path):
        return None
    z = np.load(path)
    w = z["weights"] if "weights" in z.files else None
    hubs = z["hubs"] if "hubs" in z.files else None
    return CSR(n=int(z["offsets"].shape[0]) - 1, offsets=z["offsets"], indices=z["indices"],
               weights=w, symmetric=symmetrize, hubs=hubs, name=name, key=key)


def _cache_store(g: CSR) -> None:
    cdir = os.environ.get(CACHE_ENV)
    if not cdir or not g.key:
        return
    os.makedirs(cdir, exist_ok=True)
    arrays = {"offsets": g.offsets, "indices": g.indices}
    if g.weights is not None:
        arrays["weights"] = g.weights
    if g.hubs is not None:
        arrays["hubs"] = g.hubs
    tmp = os.path.join(cdir, f"{g.key}.tmp{os.getpid()}.npz")
    np.savez(tmp, **arrays)
    os.replace(tmp, os.path.join(cdir, g.key + ".npz"))


def rmat(scale: int, nsamples: int, seed: int, *, symmetrize: bool, weighted: bool = False,
         wmin: int = 1, wmax: int = 100, n_hubs: int = 0, hub_degree: int = 0,
         a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C, nthreads: int = 0,
         name: str = "") -> CSR:
    """RMAT graph with self-loops and duplicate entries removed (see module docstring)."""
    key = _recipe_key(scale=scale, nsamples=nsamples, seed=seed, symmetrize=bool(symmetrize),
                      weighted=bool(weighted), wmin=wmin, wmax=wmax, n_hubs=n_hubs,
                      hub_degree=hub_degree, a=a, b=b, c=c)
    cached = _cache_load(key, name, symmetrize)
    if cached is not None:
        return cached
    lib = _load()
    p = _Params(scale, int(symmetrize), nsamples, seed, a, b, c, n_hubs, hub_degree,
                int(weighted), wmin, wmax, nthreads)
    h = ctypes.c_void_p()
    rc = lib.gg_rmat(ctypes.byref(p), ctypes.byref(h))
    if rc != 0:
        raise RuntimeError(f"graph generation failed (code {rc})")
    try:
        n = lib.gg_n(h)
        m = lib.gg_m(h)
        off = np.empty(n + 1, dtype=np.uint32)
        idx = np.empty(m, dtype=np.uint32)
        w = np.empty(m, dtype=np.uint32) if weighted else None
        hubs = np.empty(lib.gg_num_hubs(h), dtype=np.uint32)
        lib.gg_copy(h, off.ctypes.data, idx.ctypes.data,
                    w.ctypes.data if w is not None else None,
                    hubs.ctypes.data if hubs.size else None)
    finally:
        lib.gg_free(h)
    g = CSR(n=n, offsets=off, indices=idx, weights=w, symmetric=symmetrize,
            hubs=hubs if hubs.size else None, name=name, key=key)
    _cache_store(g)
    return g


def edge_weight(seed: int, u: int, v: int, wmin: int = 1, wmax: int = 100) -> int:
    return int(_load().gg_edge_weight(seed, u, v, wmin, wmax))


# --- the three single-graph workloads -------------------------------------------------------

def rmat16_directed(nthreads: int = 0) -> CSR:
    return rmat(16, 16 << 16, 1, symmetrize=False, nthreads=nthreads, name="rmat16-directed")


def rmat22_sym(nthreads: int = 0) -> CSR:
    return rmat(22, 16 << 22, 2, symmetrize=True, weighted=True, nthreads=nthreads,
                name="rmat22-sym-w")


def rmat24_hubs_sym(nthreads: int = 0) -> CSR:
    return rmat(24, 16 << 24, 3, symmetrize=True, weighted=True, n_hubs=16,
                hub_degree=1 << 22, nthreads=nthreads, name="rmat24-16hubs-sym-w")


def scaled_hub_graph(scale: int, seed: int = 3, n_hubs: int = 16, hub_shift: int = 2,
                     nthreads: int = 0) -> CSR:
    """Smaller member of the severe-imbalance family: hubs of degree n / 2^hub_shift."""
    return rmat(scale, 16 << scale, seed, symmetrize=True, weighted=True, n_hubs=n_hubs,
                hub_degree=(1 << scale) >> hub_shift, nthreads=nthreads,
                name=f"rmat{scale}-{n_hubs}hubs-sym-w")


def small_graph_sizes(count: int = 512, seed: int = 4) -> list[tuple[int, int]]:
    """(scale, nsamples) of the many-small-graphs batch: samples log-uniform in [2^10, 2^22]."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    out = []
    for _ in range(count):
        u = rng.uniform(10.0, 22.0)
        ms = int(math.floor(2.0 ** u))
        sc = max(4, int(round(math.log2(ms / 16.0))))
        out.append((sc, ms))
    return out


# --- tiny hand-built graphs -----------------------------------------------------------------

def from_edges(n: int, edges, weights=None, *, symmetrize: bool = False, dedup: bool = True,
               drop_self_loops: bool = True, name: str = "") -> CSR:
    """CSR from an explicit edge list (test fixtures). Weights follow their edge."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    w = None if weights is None else np.asarray(list(weights), dtype=np.int64).reshape(-1)
    if symmetrize and e.size:
        e = np.concatenate([e, e[:, ::-1]])
        if w is not None:
            w = np.concatenate([w, w])
    if drop_self_loops and e.size:
        keep = e[:, 0] != e[:, 1]
        e = e[keep]
        if w is not None:
            w = w[keep]
    if e.size:
        order = np.lexsort((e[:, 1], e[:, 0]))
        e = e[order]
        if w is not None:
            w = w[order]
        if dedup:
            keep = np.ones(len(e), dtype=bool)
            keep[1:] = np.any(e[1:] != e[:-1], axis=1)
            e = e[keep]
            if w is not None:
                w = w[keep]
    src = e[:, 0] if e.size else np.zeros(0, dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    idx = (e[:, 1] if e.size else np.zeros(0, dtype=np.int64)).astype(np.uint32)
    return CSR(n=n, offsets=off.astype(np.uint32), indices=idx,
               weights=None if w is None else w.astype(np.uint32), symmetric=symmetrize, name=name)


def random_graph(n: int, m: int, seed: int, *, symmetrize: bool, weighted: bool = True,
                 wmax: int = 100) -> CSR:
    """Uniform random multigraph fixture (dedup'd), for small parity cases."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    src = rng.integers(0, max(n, 1), size=m)
    dst = rng.integers(0, max(n, 1), size=m)
    w = rng.integers(1, wmax + 1, size=m) if weighted else None
    g = from_edges(n, np.stack([src, dst], axis=1) if m else [], w, symmetrize=False)
    if symmetrize:
        # symmetric weights: the weight of {u, v} is the one of its smaller-first orientation
        e = np.stack([np.repeat(np.arange(n), np.diff(g.offsets.astype(np.int64))),
                      g.indices.astype(np.int64)], axis=1)
        ww = None
        if weighted:
            lo = np.minimum(e[:, 0], e[:, 1]); hi = np.maximum(e[:, 0], e[:, 1])
            ww = (((lo * 1000003 + hi * 7919 + seed) % wmax) + 1)
        g = from_edges(n, e, ww, symmetrize=True)
    return g


def disjoint_union(graphs: list[CSR], name: str = "") -> tuple[CSR, np.ndarray]:
    """One CSR holding every graph of `graphs`, graph i's vertex v renumbered to base[i] + v.

    Returns (union, base) with base[i] the first vertex id of graph i (base[-1] = total n).
    Traversals of the union from one source per graph give each graph's own result.
    """
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    ms = np.array([g.m for g in graphs], dtype=np.int64)
    base = np.concatenate([[0], np.cumsum(ns)])
    ebase = np.concatenate([[0], np.cumsum(ms)])
    if base[-1] >= 2 ** 32 - 1 or ebase[-1] >= 2 ** 32 - 1:
        raise ValueError("union too large for uint32 CSR")
    off = np.empty(int(base[-1]) + 1, dtype=np.uint32)
    idx = np.empty(int(ebase[-1]), dtype=np.uint32)
    weighted = all(g.weights is not None for g in graphs)
    w = np.empty(int(ebase[-1]), dtype=np.uint32) if weighted else None
    for i, g in enumerate(graphs):
        off[base[i]:base[i + 1]] = g.offsets[:-1].astype(np.int64) + ebase[i]
        idx[ebase[i]:ebase[i + 1]] = g.indices.astype(np.int64) + base[i]
        if weighted:
            w[ebase[i]:ebase[i + 1]] = g.weights
    off[-1] = ebase[-1]
    return CSR(n=int(base[-1]), offsets=off, indices=idx, weights=w,
               symmetric=all(g.symmetric for g in graphs), name=name), base


def small_graphs(count: int = 512, seed: int = 4, nthreads: int = 0) -> list[CSR]:
    """The many-small-graphs batch: RMAT graphs whose sample counts are log-uniform in
    [2^10, 2^22] (scale = max(4, round(log2(samples / 16)))), symmetrised, weights 1..100,
    graph i drawn with seed 1000 * seed + i."""
    out = []
    for i, (sc, ms) in enumerate(small_graph_sizes(count, seed)):
        out.append(rmat(sc, ms, 1000 * seed + i, symmetrize=True, weighted=True, nthreads=nthreads,
                        name=f"small{i}"))
    return out
