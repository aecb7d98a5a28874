"""The allocation-free BFS entry point against the regular one.

alb_bfs_noalloc exists for callers that may not allocate device memory (code
that runs while a CUDA graph is being captured, services whose device memory
belongs to another allocator, loops that must never block in cudaMalloc). It
must give exactly what alb_bfs gives, call after call, although every call
reuses the same fixed scratch array inside the library.

This file is collected last on purpose; it also passes when run on its own.
"""
import numpy as np
import pytest

from paper_1911_09135_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_09135_gb300 import alb  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def reference_levels(g, d_off, d_idx, src):
    """Levels from the regular entry point (graph handle, library-owned workspace)."""
    with alb.Graph(g.n, d_off, d_idx, symmetric=g.symmetric) as G:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        G.bfs(src, out)
        G.sync()
        return out.clone()


@pytest.mark.parametrize("which", ["rmat16-directed", "rmat20-sym-max-size"])
def test_noalloc_bfs_equals_alb_bfs_twice(which):
    if which == "rmat16-directed":
        g = gg.rmat16_directed()
        sources = [0, 40000]
    else:
        g = gg.rmat(20, 16 << 20, 8, symmetrize=True)  # n = 2^20, the largest accepted
        sources = [g.max_degree_vertex(), 12345]
    assert g.n <= alb.ALB_NOALLOC_MAX_VERTICES
    d_off, d_idx = dev(g.offsets), dev(g.indices)
    out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    # two calls in a row: the second starts from the first call's leftovers in the scratch
    for src in sources:
        alb.alb_bfs_noalloc(g.n, g.m, d_off, d_idx, src, out)
        torch.cuda.synchronize()
        assert torch.equal(out, reference_levels(g, d_off, d_idx, src)), src


def test_noalloc_rejects_graphs_above_the_limit():
    n = alb.ALB_NOALLOC_MAX_VERTICES + 1
    d_off = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(alb.AlbError) as e:
        alb.alb_bfs_noalloc(n, 0, d_off, None, 0, out)
    assert e.value.code == 1  # ALB_ERR_INVALID_ARG, nothing enqueued
