"""In-tree build of the package's native libraries.

* ``libalbgen.so``  - the seeded graph generator (host C++/OpenMP).
* ``libalb.so``     - the CUDA kernels and the C ABI declared in ``include/alb.h``,
                      compiled for sm_103a only.

Everything is compiled with plain ``g++``/``nvcc`` command lines (no cmake), the
CUDA translation units in parallel, so a fresh build takes about a minute.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os
import shutil
import subprocess
import sys

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
LIB_DIR = os.path.join(PKG_DIR, "_lib")
OBJ_DIR = os.path.join(REPO_DIR, "_build", "alb")
INCLUDE_DIR = os.path.join(REPO_DIR, "include")

GENCODE = "-gencode=arch=compute_103a,code=sm_103a"

ALB_SOURCES = [
    "alb/alb_graph.cu",
    "alb/alb_traverse.cu",
    "alb/alb_pagerank.cu",
    "alb/alb_batch.cu",
    "alb/alb_tune.cu",
    "alb/alb_partition.cu",
]
ALB_HEADERS = [
    "alb/alb_internal.cuh",
    "alb/alb_device.cuh",
    "alb/alb_kernels.cuh",
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libalb.so")


def _run(cmd: list[str]) -> None:
    proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build command failed:\n" + " ".join(cmd) + "\n" + proc.stdout)


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps if os.path.exists(d))


def build_graphgen(force: bool = False) -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    src = os.path.join(CSRC, "gen", "graphgen.cpp")
    out = os.path.join(LIB_DIR, "libalbgen.so")
    if force or not _newer(out, [src]):
        tmp = out + ".tmp%d" % os.getpid()
        _run(["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, out)
    return out


def build_alb(force: bool = False, extra_flags: list[str] | None = None, checked: bool = False) -> str:
    """libalb.so; checked=True builds libalb_checked.so (-DALB_CHECKED: bounds-checked kernels)."""
    obj_dir = OBJ_DIR + ("_checked" if checked else "")
    os.makedirs(LIB_DIR, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    out = os.path.join(LIB_DIR, "libalb_checked.so" if checked else "libalb.so")
    if checked:
        extra_flags = list(extra_flags or []) + ["-DALB_CHECKED"]
    headers = [os.path.join(CSRC, h) for h in ALB_HEADERS] + [os.path.join(INCLUDE_DIR, "alb.h")]
    nvcc = _nvcc()
    flags = [
        GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
        "-I" + INCLUDE_DIR, "-I" + os.path.join(CSRC, "alb"),
    ] + list(extra_flags or [])

    def compile_one(rel: str) -> str:
        src = os.path.join(CSRC, rel)
        obj = os.path.join(obj_dir, os.path.basename(rel) + ".o")
        if force or not _newer(obj, [src] + headers + [__file__]):
            _run([nvcc, "-c", src, "-o", obj] + flags)
        return obj

    with _cf.ThreadPoolExecutor(max_workers=min(8, len(ALB_SOURCES))) as ex:
        objs = list(ex.map(compile_one, ALB_SOURCES))
    if force or not _newer(out, objs):
        tmp = out + ".tmp%d" % os.getpid()
        _run([nvcc, GENCODE, "-shared", "-o", tmp] + objs)
        os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> None:
    build_graphgen(force)
    build_alb(force)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
