"""CPU oracle (test infrastructure only).

ctypes binding of ``oracle/oracle.c``: plain, serial, obviously correct
definitions of what the ALB path computes (arXiv:1911.09135, Sec. 4 and 5).
Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the library in ``paper_1911_09135_gb300`` never imports it, and it
imports nothing from there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "liboracle.so")
INF = 0xFFFFFFFF

OR_OK, OR_ERR_ARG, OR_ERR_OOM, OR_ERR_OVERFLOW, OR_ERR_CHECK = range(5)


def build(force: bool = False) -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
        proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if proc.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + proc.stdout)
        os.replace(tmp, LIB)
    return LIB


_lib = None
_P = ctypes.c_void_p
_U32 = ctypes.c_uint32


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_bfs.argtypes = [_U32, _P, _P, _U32, _P]
        lib.oracle_sssp.argtypes = [_U32, _P, _P, _P, _U32, _P]
        lib.oracle_cc.argtypes = [_U32, _P, _P, _P]
        lib.oracle_pagerank.argtypes = [_U32, _P, _P, ctypes.c_double, ctypes.c_double, _U32,
                                        ctypes.c_int, ctypes.c_int, _P, _P, _P]
        lib.oracle_kcore.argtypes = [_U32, _P, _P, _U32, _P]
        lib.oracle_inspect.argtypes = [_U32, _P, _P, _U32, _U32, _U32, _U32, _P, _P, _P, _P]
        lib.oracle_lb_edges.argtypes = [_P, _P, _P, _P, _U32, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_int, _P, _P, _P, ctypes.c_int64]
        lib.oracle_lb_edges.restype = ctypes.c_int64
        lib.oracle_check_bfs.argtypes = [_U32, _P, _P, _U32, _P, _P]
        lib.oracle_check_sssp.argtypes = [_U32, _P, _P, _P, _U32, _P, _P]
        for f in ("oracle_bfs", "oracle_sssp", "oracle_cc", "oracle_pagerank", "oracle_kcore",
                  "oracle_inspect", "oracle_check_bfs", "oracle_check_sssp"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str) -> None:
    if rc != OR_OK:
        raise OracleError(f"{what} failed with code {rc}")


# On-disk cache of results on large graphs: with ALB_ORACLE_CACHE set to a directory, a call that
# names its graph by `cache_key` (a digest of how the graph was made, e.g. the generator's recipe
# key) stores its result there under (function, key, arguments, digest of oracle.c) and later calls
# read it back instead of recomputing (a scale-24 Dijkstra or PageRank takes tens of seconds).
# Calls without a key are never cached.
CACHE_ENV = "ALB_ORACLE_CACHE"


def _cached(fn: str, cache_key, args: tuple, compute):
    cdir = os.environ.get(CACHE_ENV)
    if not cdir or not cache_key:
        return compute()
    import hashlib
    h = hashlib.sha256(open(SRC, "rb").read())
    h.update(repr((fn, cache_key, args)).encode())
    path = os.path.join(cdir, "oracle-" + h.hexdigest()[:32] + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        vals = [z[f"r{i}"] for i in range(len(z.files))]
        vals = [v.item() if v.ndim == 0 else v for v in vals]
        return vals[0] if len(vals) == 1 else tuple(vals)
    res = compute()
    os.makedirs(cdir, exist_ok=True)
    parts = res if isinstance(res, tuple) else (res,)
    tmp = path[:-4] + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **{f"r{i}": np.asarray(v) for i, v in enumerate(parts)})
    os.replace(tmp, path)
    return res


def bfs(n, offsets, indices, src, *, cache_key=None) -> np.ndarray:
    def run():
        off, idx = _u32(offsets), _u32(indices)
        out = np.empty(n, dtype=np.uint32)
        _check(_load().oracle_bfs(n, _ptr(off), _ptr(idx), src, _ptr(out)), "oracle_bfs")
        return out
    return _cached("bfs", cache_key, (n, src), run)


def sssp(n, offsets, indices, weights, src, *, cache_key=None) -> np.ndarray:
    def run():
        off, idx, w = _u32(offsets), _u32(indices), _u32(weights)
        out = np.empty(n, dtype=np.uint32)
        _check(_load().oracle_sssp(n, _ptr(off), _ptr(idx), _ptr(w), src, _ptr(out)), "oracle_sssp")
        return out
    return _cached("sssp", cache_key, (n, src), run)


def cc(n, offsets, indices, *, cache_key=None) -> np.ndarray:
    def run():
        off, idx = _u32(offsets), _u32(indices)
        out = np.empty(n, dtype=np.uint32)
        _check(_load().oracle_cc(n, _ptr(off), _ptr(idx), _ptr(out)), "oracle_cc")
        return out
    return _cached("cc", cache_key, (n,), run)


def pagerank(n, offsets, indices, damping=0.85, tol=1e-6, max_iter=1000, *,
             assume_symmetric=False, nthreads=0, cache_key=None):
    """Returns (x float64[n], iterations, last L1 change)."""
    def run():
        off, idx = _u32(offsets), _u32(indices)
        x = np.empty(max(n, 1), dtype=np.float64)
        it = ctypes.c_uint32(0)
        l1 = ctypes.c_double(0.0)
        _check(_load().oracle_pagerank(n, _ptr(off), _ptr(idx), damping, tol, max_iter,
                                       int(assume_symmetric), nthreads, _ptr(x), ctypes.byref(it),
                                       ctypes.byref(l1)), "oracle_pagerank")
        return x[:n], int(it.value), float(l1.value)
    # the thread count does not change the result (each vertex's sum is sequential)
    x, it, l1 = _cached("pagerank", cache_key, (n, damping, tol, max_iter, bool(assume_symmetric)), run)
    return x, int(it), float(l1)


def kcore(n, offsets, indices, k, *, cache_key=None) -> np.ndarray:
    def run():
        off, idx = _u32(offsets), _u32(indices)
        out = np.empty(n, dtype=np.uint32)
        _check(_load().oracle_kcore(n, _ptr(off), _ptr(idx), k, _ptr(out)), "oracle_kcore")
        return out
    return _cached("kcore", cache_key, (n, k), run)


def inspect(n, offsets, worklist, threshold, warp_min=32, cta_min=256):
    """Algorithm 1. Returns (work uint32[v], prefix uint64[v+1], bin uint8[nf], counts[4])."""
    off, wl = _u32(offsets), _u32(worklist)
    nf = int(wl.shape[0])
    work = np.empty(max(nf, 1), dtype=np.uint32)
    prefix = np.empty(nf + 1, dtype=np.uint64)
    b = np.empty(max(nf, 1), dtype=np.uint8)
    counts = np.zeros(4, dtype=np.uint32)
    _check(_load().oracle_inspect(n, _ptr(off), _ptr(wl), nf, threshold, warp_min, cta_min,
                                  _ptr(work), _ptr(prefix), _ptr(b), _ptr(counts)),
           "oracle_inspect")
    v = int(counts[3])
    return work[:v].copy(), prefix[:v + 1].copy(), b[:nf].copy(), counts


def lb_edges(offsets, indices, work, prefix, p, i, policy="cyclic"):
    """Algorithm 2 for thread i of p. Returns (k uint64[], src uint32[], dst uint32[])."""
    off, idx, wk = _u32(offsets), _u32(indices), _u32(work)
    pre = np.ascontiguousarray(prefix, dtype=np.uint64)
    pol = 0 if policy == "cyclic" else 1
    nwork = int(wk.shape[0])
    lib = _load()
    cnt = lib.oracle_lb_edges(_ptr(off), _ptr(idx), _ptr(wk), _ptr(pre), nwork, p, i, pol,
                              None, None, None, 0)
    ks = np.empty(max(cnt, 1), dtype=np.uint64)
    ss = np.empty(max(cnt, 1), dtype=np.uint32)
    ds = np.empty(max(cnt, 1), dtype=np.uint32)
    lib.oracle_lb_edges(_ptr(off), _ptr(idx), _ptr(wk), _ptr(pre), nwork, p, i, pol,
                        _ptr(ks), _ptr(ss), _ptr(ds), cnt)
    return ks[:cnt], ss[:cnt], ds[:cnt]


def check_bfs(n, offsets, indices, src, level) -> int:
    """-1 if `level` is exactly the BFS level array from src, else a failing vertex."""
    off, idx, lv = _u32(offsets), _u32(indices), _u32(level)
    bad = ctypes.c_int64(-1)
    rc = _load().oracle_check_bfs(n, _ptr(off), _ptr(idx), src, _ptr(lv), ctypes.byref(bad))
    if rc not in (OR_OK, OR_ERR_CHECK):
        raise OracleError(f"oracle_check_bfs failed with code {rc}")
    return -1 if rc == OR_OK else max(int(bad.value), 0)


def check_sssp(n, offsets, indices, weights, src, dist) -> int:
    """-1 if `dist` is exactly the shortest-path distance array from src, else a failing vertex."""
    off, idx, w, d = _u32(offsets), _u32(indices), _u32(weights), _u32(dist)
    bad = ctypes.c_int64(-1)
    rc = _load().oracle_check_sssp(n, _ptr(off), _ptr(idx), _ptr(w), src, _ptr(d),
                                   ctypes.byref(bad))
    if rc not in (OR_OK, OR_ERR_CHECK):
        raise OracleError(f"oracle_check_sssp failed with code {rc}")
    return -1 if rc == OR_OK else max(int(bad.value), 0)
