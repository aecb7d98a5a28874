"""Python binding of libalb.so (include/alb.h): argument marshalling only.

Every step of every traversal runs in the library's CUDA kernels. Arrays may be
torch CUDA tensors (device memory) or numpy arrays / CPU tensors (host memory);
the library detects which, exactly as the C ABI documents. Streams are torch
streams (or raw ``cudaStream_t`` integers); ``None`` means torch's current
stream when torch is importable, else the legacy default stream.

There is no CPU fallback: if ``libalb.so`` cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

ALB_UNREACHED = 0xFFFFFFFF
ALB_SYMMETRIC = 0x1
ALB_VALIDATE = 0x2

STATUS = {
    0: "ALB_OK", 1: "ALB_ERR_INVALID_ARG", 2: "ALB_ERR_OOM", 3: "ALB_ERR_CUDA",
    4: "ALB_ERR_TIMEOUT", 5: "ALB_ERR_OVERFLOW", 6: "ALB_ERR_NOT_SYMMETRIC",
    7: "ALB_ERR_UNSUPPORTED", 8: "ALB_ERR_DEVICE",
}

# Every entry point declared in include/alb.h.
EXPORTS = [
    "alb_graph_create", "alb_graph_destroy", "alb_default_params", "alb_set_params",
    "alb_get_params", "alb_bfs", "alb_sssp", "alb_cc", "alb_pagerank", "alb_kcore",
    "alb_bfs_batch", "alb_sssp_batch", "alb_inspect", "alb_lb_trace", "alb_threshold_rule",
    "alb_sync", "alb_get_stats", "alb_status_str", "alb_version", "alb_bfs_noalloc",
    "alb_bfs_multi", "alb_sssp_multi", "alb_autotune", "alb_set_app_params", "alb_get_app_params",
    "alb_graph_clone", "alb_debug_check", "alb_checked_build", "alb_get_cta_loads",
    "alb_partition_split", "alb_partition_sms", "alb_partition_stream_create",
    "alb_partition_stream_destroy", "alb_partition_destroy", "alb_graph_trim",
]

ALB_APP = {"bfs": 0, "sssp": 1, "cc": 2, "pr": 3, "pagerank": 3, "kcore": 4}


class AlbError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class alb_params(ctypes.Structure):
    _fields_ = [
        ("hub_threshold", ctypes.c_int64),
        ("twc_warp_min", ctypes.c_uint32),
        ("twc_cta_min", ctypes.c_uint32),
        ("grid_blocks", ctypes.c_uint32),
        ("distribution", ctypes.c_uint32),
        ("exec_mode", ctypes.c_uint32),
        ("max_rounds", ctypes.c_uint32),
        ("l2_persist_fraction", ctypes.c_float),
        ("profile", ctypes.c_uint32),
        ("cta_stats", ctypes.c_uint32),
        ("block_size", ctypes.c_uint32),
    ]


class alb_stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32), ("hub_rounds", ctypes.c_uint32),
        ("max_hub_count", ctypes.c_uint32), ("hub_threshold", ctypes.c_uint32),
        ("lb_threads", ctypes.c_uint32), ("grid_blocks", ctypes.c_uint32),
        ("block_size", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
        ("edges_twc", ctypes.c_uint64), ("edges_lb", ctypes.c_uint64),
        ("pushes", ctypes.c_uint64), ("pr_l1", ctypes.c_double),
        ("ms_inspect", ctypes.c_double), ("ms_lb", ctypes.c_double), ("ms_other", ctypes.c_double),
        ("n_inspect", ctypes.c_uint32), ("n_lb", ctypes.c_uint32), ("n_other", ctypes.c_uint32),
        ("reserved2", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


_lib = None
_P = ctypes.c_void_p
_U32 = ctypes.c_uint32


def lib_path() -> str:
    """libalb.so, or the bounds-checked libalb_checked.so when ALB_CHECKED=1 is set."""
    name = "libalb_checked.so" if os.environ.get("ALB_CHECKED") == "1" else "libalb.so"
    return os.path.join(_build.LIB_DIR, name)


def load(build_if_missing: bool = False):
    """Load libalb.so (raises if it is missing and not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} not found; build it with paper_1911_09135_gb300._build.build_alb()")
        path = _build.build_alb(checked=os.environ.get("ALB_CHECKED") == "1")
    lib = ctypes.CDLL(path)
    S = ctypes.c_int
    sig = {
        "alb_graph_create": ([_U32, ctypes.c_uint64, _P, _P, _P, _U32, _P, ctypes.POINTER(_P)], S),
        "alb_graph_destroy": ([_P], S),
        "alb_graph_clone": ([_P, ctypes.POINTER(_P)], S),
        "alb_graph_trim": ([_P, ctypes.POINTER(ctypes.c_uint64)], S),
        "alb_debug_check": ([_P, _P], S),
        "alb_get_cta_loads": ([_P, _P, _P, _U32, ctypes.POINTER(_U32), ctypes.POINTER(_U32)], S),
        "alb_checked_build": ([], _U32),
        "alb_default_params": ([ctypes.POINTER(alb_params)], S),
        "alb_set_params": ([_P, ctypes.POINTER(alb_params)], S),
        "alb_get_params": ([_P, ctypes.POINTER(alb_params)], S),
        "alb_bfs": ([_P, _U32, _P, _P], S),
        "alb_sssp": ([_P, _U32, _P, _P], S),
        "alb_cc": ([_P, _P, _P], S),
        "alb_pagerank": ([_P, ctypes.c_float, ctypes.c_double, _U32, _P, _P, _P, _P], S),
        "alb_kcore": ([_P, _U32, _P, _P], S),
        "alb_bfs_batch": ([_P, _P, _U32, _P, _P], S),
        "alb_sssp_batch": ([_P, _P, _U32, _P, _P], S),
        "alb_bfs_multi": ([_P, _P, _U32, _P, _P], S),
        "alb_set_app_params": ([_P, S, ctypes.POINTER(alb_params)], S),
        "alb_get_app_params": ([_P, S, ctypes.POINTER(alb_params)], S),
        "alb_autotune": ([_P, S, _U32, _U32, ctypes.POINTER(alb_params), ctypes.POINTER(ctypes.c_float), _P], S),
        "alb_sssp_multi": ([_P, _P, _U32, _P, _P], S),
        "alb_inspect": ([_P, _P, _U32, _P, _P, _P, _P, _P], S),
        "alb_lb_trace": ([_P, _P, _P, _U32, _P, _P, _P, _P], S),
        "alb_threshold_rule": ([_U32, _U32], _U32),
        "alb_sync": ([_P], S),
        "alb_get_stats": ([_P, ctypes.POINTER(alb_stats)], S),
        "alb_status_str": ([S], ctypes.c_char_p),
        "alb_version": ([], _U32),
        "alb_bfs_noalloc": ([_U32, ctypes.c_uint64, _P, _P, _U32, _P, _P], S),
        "alb_partition_split": ([S, _U32, ctypes.POINTER(_P), ctypes.POINTER(_P)], S),
        "alb_partition_sms": ([_P, ctypes.POINTER(_U32)], S),
        "alb_partition_stream_create": ([_P, S, ctypes.POINTER(_P)], S),
        "alb_partition_stream_destroy": ([_P], S),
        "alb_partition_destroy": ([_P], S),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise AlbError(rc, what)


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _dtype_ok(a, kind: str) -> bool:
    name = str(a.dtype)
    return {"u32": ("uint32", "torch.uint32", "int32", "torch.int32"),
            "f32": ("float32", "torch.float32"), "f64": ("float64", "torch.float64"),
            "u8": ("uint8", "torch.uint8")}[kind].__contains__(name)


def _want(a, n: int, kind: str, what: str) -> None:
    if _numel(a) < n or not _dtype_ok(a, kind):
        raise ValueError(f"{what}: need >= {n} elements of {kind}, got {a.dtype} x {_numel(a)}")


# ----------------------------------------------------------------- C-ABI mirrors

def alb_graph_create(n, m, offsets, indices, weights=None, flags=0, stream=None) -> int:
    lib = load()
    _want(offsets, n + 1, "u32", "offsets")
    if m:
        _want(indices, m, "u32", "indices")
    if weights is not None:
        _want(weights, m, "u32", "weights")
    h = _P()
    _check(lib.alb_graph_create(n, m, _ptr(offsets), _ptr(indices), _ptr(weights), flags,
                                _stream(stream), ctypes.byref(h)), "alb_graph_create")
    return h.value


def alb_graph_clone(g) -> int:
    h = _P()
    _check(load().alb_graph_clone(g, ctypes.byref(h)), "alb_graph_clone")
    return h.value


def alb_graph_destroy(g) -> None:
    _check(load().alb_graph_destroy(g), "alb_graph_destroy")


def alb_graph_trim(g) -> int:
    """Release the handle's cached per-call workspaces; returns the bytes the device got back."""
    freed = ctypes.c_uint64(0)
    _check(load().alb_graph_trim(g, ctypes.byref(freed)), "alb_graph_trim")
    return int(freed.value)


def alb_default_params() -> alb_params:
    p = alb_params()
    _check(load().alb_default_params(ctypes.byref(p)), "alb_default_params")
    return p


def alb_set_params(g, p: alb_params) -> None:
    _check(load().alb_set_params(g, ctypes.byref(p)), "alb_set_params")


def alb_get_params(g) -> alb_params:
    p = alb_params()
    _check(load().alb_get_params(g, ctypes.byref(p)), "alb_get_params")
    return p


def alb_set_app_params(g, app, p: alb_params) -> None:
    code = ALB_APP[app] if isinstance(app, str) else int(app)
    _check(load().alb_set_app_params(g, code, ctypes.byref(p)), "alb_set_app_params")


def alb_get_app_params(g, app) -> alb_params:
    p = alb_params()
    code = ALB_APP[app] if isinstance(app, str) else int(app)
    _check(load().alb_get_app_params(g, code, ctypes.byref(p)), "alb_get_app_params")
    return p


def alb_bfs(g, src, levels, stream=None) -> None:
    _check(load().alb_bfs(g, src, _ptr(levels), _stream(stream)), "alb_bfs")


def alb_sssp(g, src, dist, stream=None) -> None:
    _check(load().alb_sssp(g, src, _ptr(dist), _stream(stream)), "alb_sssp")


def alb_cc(g, labels, stream=None) -> None:
    _check(load().alb_cc(g, _ptr(labels), _stream(stream)), "alb_cc")


def alb_pagerank(g, damping, tol, max_iter, rank, l1=None, iters=None, stream=None) -> None:
    _check(load().alb_pagerank(g, damping, tol, max_iter, _ptr(rank), _ptr(l1), _ptr(iters),
                               _stream(stream)), "alb_pagerank")


def alb_kcore(g, k, in_core, stream=None) -> None:
    _check(load().alb_kcore(g, k, _ptr(in_core), _stream(stream)), "alb_kcore")


def alb_bfs_batch(g, srcs, k, out, stream=None) -> None:
    _check(load().alb_bfs_batch(g, _ptr(srcs), k, _ptr(out), _stream(stream)), "alb_bfs_batch")


def alb_sssp_batch(g, srcs, k, out, stream=None) -> None:
    _check(load().alb_sssp_batch(g, _ptr(srcs), k, _ptr(out), _stream(stream)), "alb_sssp_batch")


def alb_bfs_multi(g, srcs, k, levels, stream=None) -> None:
    _check(load().alb_bfs_multi(g, _ptr(srcs), k, _ptr(levels), _stream(stream)), "alb_bfs_multi")


def alb_sssp_multi(g, srcs, k, dist, stream=None) -> None:
    _check(load().alb_sssp_multi(g, _ptr(srcs), k, _ptr(dist), _stream(stream)), "alb_sssp_multi")


def alb_autotune(g, app, src=0, reps=3, stream=None):
    """Returns (best alb_params, best time in ms); the best setting is left applied."""
    p = alb_params()
    ms = ctypes.c_float(0.0)
    code = ALB_APP[app] if isinstance(app, str) else int(app)
    _check(load().alb_autotune(g, code, src, reps, ctypes.byref(p), ctypes.byref(ms), _stream(stream)),
           "alb_autotune")
    return p, float(ms.value)


def alb_inspect(g, wl, nf, bins, work, prefix, counts, stream=None) -> None:
    _check(load().alb_inspect(g, _ptr(wl), nf, _ptr(bins), _ptr(work), _ptr(prefix),
                              _ptr(counts), _stream(stream)), "alb_inspect")


def alb_lb_trace(g, work, prefix, nwork, src, dst, thread, stream=None) -> None:
    _check(load().alb_lb_trace(g, _ptr(work), _ptr(prefix), nwork, _ptr(src), _ptr(dst),
                               _ptr(thread), _stream(stream)), "alb_lb_trace")


def alb_threshold_rule(num_sms: int, threads_per_sm: int) -> int:
    return int(load().alb_threshold_rule(num_sms, threads_per_sm))


def alb_sync(g) -> None:
    _check(load().alb_sync(g), "alb_sync")


def alb_get_stats(g) -> alb_stats:
    s = alb_stats()
    _check(load().alb_get_stats(g, ctypes.byref(s)), "alb_get_stats")
    return s


def alb_status_str(code: int) -> str:
    return load().alb_status_str(code).decode()


def alb_version() -> int:
    return int(load().alb_version())


def alb_get_cta_loads(g, cap: int = 1 << 16):
    """(twc, lb): per-CTA edge counts of the last cta_stats call, as uint64 arrays."""
    twc = np.zeros(cap, dtype=np.uint64)
    lb = np.zeros(cap, dtype=np.uint64)
    nt, nl = _U32(0), _U32(0)
    _check(load().alb_get_cta_loads(g, twc.ctypes.data, lb.ctypes.data, cap, ctypes.byref(nt),
                                    ctypes.byref(nl)), "alb_get_cta_loads")
    return twc[:min(cap, nt.value)], lb[:min(cap, nl.value)]


class Partition:
    """An SM partition (alb_partition_split): streams made from it run kernels on its SMs only."""

    def __init__(self, handle: int):
        self.h = handle
        self._streams = []

    @property
    def sms(self) -> int:
        n = _U32(0)
        _check(load().alb_partition_sms(self.h, ctypes.byref(n)), "alb_partition_sms")
        return int(n.value)

    def stream(self, priority: int = 0) -> int:
        """A new non-blocking stream of the partition (a cudaStream_t as int), owned by it."""
        s = _P()
        _check(load().alb_partition_stream_create(self.h, priority, ctypes.byref(s)),
               "alb_partition_stream_create")
        self._streams.append(s.value)
        return int(s.value)

    def close(self):
        for s in self._streams:
            load().alb_partition_stream_destroy(s)
        self._streams = []
        if self.h:
            load().alb_partition_destroy(self.h)
            self.h = None


def partition_split(device: int, sm_count: int):
    """(first, rest): device split into sm_count SMs (rounded up) and the remaining SMs."""
    a, b = _P(), _P()
    _check(load().alb_partition_split(device, sm_count, ctypes.byref(a), ctypes.byref(b)),
           "alb_partition_split")
    return Partition(a.value), Partition(b.value)


def alb_checked_build() -> int:
    return int(load().alb_checked_build())


def alb_debug_check(g) -> list[int]:
    out = np.zeros(4, dtype=np.uint32)
    _check(load().alb_debug_check(g, out.ctypes.data), "alb_debug_check")
    return out.tolist()


ALB_NOALLOC_MAX_VERTICES = 1 << 20


def alb_bfs_noalloc(n, m, offsets, indices, src, levels, stream=None) -> None:
    """BFS that allocates nothing (see include/alb.h): CUDA tensors in and out."""
    _check(load().alb_bfs_noalloc(n, m, _ptr(offsets), _ptr(indices), src, _ptr(levels),
                                  _stream(stream)), "alb_bfs_noalloc")


# ------------------------------------------------------------- convenience wrapper

class Graph:
    """Owns one alb_graph handle. Arrays in/out may be host numpy or CUDA tensors."""

    def __init__(self, n, offsets, indices, weights=None, symmetric=False, stream=None):
        self.n = int(n)
        self.m = _numel(indices)
        self.symmetric = symmetric
        flags = ALB_SYMMETRIC if symmetric else 0
        self.h = alb_graph_create(self.n, self.m, offsets, indices, weights, flags, stream)

    def clone(self) -> "Graph":
        """Another handle on the same device CSR with its own workspace (concurrent use)."""
        c = Graph.__new__(Graph)
        c.n, c.m, c.symmetric = self.n, self.m, self.symmetric
        c.h = alb_graph_clone(self.h)
        return c

    @classmethod
    def from_csr(cls, csr, stream=None):
        return cls(csr.n, csr.offsets, csr.indices, csr.weights, csr.symmetric, stream)

    def close(self):
        if getattr(self, "h", None):
            alb_graph_destroy(self.h)
            self.h = None

    def trim(self) -> int:
        """Release cached per-call workspaces (the CSR stays); bytes given back."""
        return alb_graph_trim(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def params(self, app=None) -> alb_params:
        return alb_get_params(self.h) if app is None else alb_get_app_params(self.h, app)

    def set_app_params(self, app, **kw) -> None:
        p = alb_get_app_params(self.h, app)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise AttributeError(k)
            setattr(p, k, v)
        alb_set_app_params(self.h, app, p)

    def set_params(self, **kw) -> None:
        p = alb_get_params(self.h)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise AttributeError(k)
            setattr(p, k, v)
        alb_set_params(self.h, p)

    def _out(self, out, dtype, count=None):
        count = self.n if count is None else count
        if out is None:
            out = np.empty(count, dtype=dtype)
        return out

    def bfs(self, src, out=None, stream=None):
        out = self._out(out, np.uint32)
        _want(out, self.n, "u32", "levels")
        alb_bfs(self.h, src, out, stream)
        return out

    def sssp(self, src, out=None, stream=None):
        out = self._out(out, np.uint32)
        _want(out, self.n, "u32", "dist")
        alb_sssp(self.h, src, out, stream)
        return out

    def cc(self, out=None, stream=None):
        out = self._out(out, np.uint32)
        _want(out, self.n, "u32", "labels")
        alb_cc(self.h, out, stream)
        return out

    def kcore(self, k, out=None, stream=None):
        out = self._out(out, np.uint32)
        _want(out, self.n, "u32", "in_core")
        alb_kcore(self.h, k, out, stream)
        return out

    def pagerank(self, damping=0.85, tol=1e-6, max_iter=1000, out=None, stream=None):
        out = self._out(out, np.float32)
        _want(out, self.n, "f32", "rank")
        l1 = np.zeros(1, dtype=np.float64)
        it = np.zeros(1, dtype=np.uint32)
        alb_pagerank(self.h, damping, tol, max_iter, out, l1, it, stream)
        return out, int(it[0]), float(l1[0])

    def bfs_batch(self, srcs, out=None, stream=None):
        srcs = np.ascontiguousarray(srcs, dtype=np.uint32) if isinstance(srcs, (list, tuple)) else srcs
        k = _numel(srcs)
        out = self._out(out, np.uint32, k * self.n)
        alb_bfs_batch(self.h, srcs, k, out, stream)
        return out

    def sssp_batch(self, srcs, out=None, stream=None):
        srcs = np.ascontiguousarray(srcs, dtype=np.uint32) if isinstance(srcs, (list, tuple)) else srcs
        k = _numel(srcs)
        out = self._out(out, np.uint32, k * self.n)
        alb_sssp_batch(self.h, srcs, k, out, stream)
        return out

    def bfs_multi(self, srcs, out=None, stream=None):
        srcs = np.ascontiguousarray(srcs, dtype=np.uint32) if isinstance(srcs, (list, tuple, np.ndarray)) else srcs
        out = self._out(out, np.uint32)
        alb_bfs_multi(self.h, srcs, _numel(srcs), out, stream)
        return out

    def sssp_multi(self, srcs, out=None, stream=None):
        srcs = np.ascontiguousarray(srcs, dtype=np.uint32) if isinstance(srcs, (list, tuple, np.ndarray)) else srcs
        out = self._out(out, np.uint32)
        alb_sssp_multi(self.h, srcs, _numel(srcs), out, stream)
        return out

    def cta_loads(self):
        return alb_get_cta_loads(self.h)

    def autotune(self, app, src=0, reps=3, stream=None):
        return alb_autotune(self.h, app, src, reps, stream)

    def inspect(self, worklist, stream=None):
        wl = np.ascontiguousarray(worklist, dtype=np.uint32)
        nf = int(wl.size)
        bins = np.zeros(max(nf, 1), dtype=np.uint8)
        work = np.zeros(nf + 1, dtype=np.uint32)
        prefix = np.zeros(nf + 1, dtype=np.uint32)
        counts = np.zeros(4, dtype=np.uint32)
        alb_inspect(self.h, wl, nf, bins, work, prefix, counts, stream)
        v = int(counts[3])
        return work[:v], prefix[:v + 1], bins[:nf], counts

    def lb_trace(self, work, prefix, stream=None):
        work = np.ascontiguousarray(work, dtype=np.uint32)
        prefix = np.ascontiguousarray(prefix, dtype=np.uint32)
        e = int(prefix[-1])
        src = np.zeros(max(e, 1), dtype=np.uint32)
        dst = np.zeros(max(e, 1), dtype=np.uint32)
        thr = np.zeros(max(e, 1), dtype=np.uint32)
        alb_lb_trace(self.h, work, prefix, int(work.size), src, dst, thr, stream)
        return src[:e], dst[:e], thr[:e]

    def sync(self):
        alb_sync(self.h)

    def stats(self) -> dict:
        return alb_get_stats(self.h).as_dict()
