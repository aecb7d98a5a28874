"""The allocation-free BFS entry point against the CPU oracle and the regular entry point.

alb_bfs_noalloc exists for callers that may not allocate device memory (code
that runs while a CUDA graph is being captured, services whose device memory
belongs to another allocator, loops that must never block in cudaMalloc). It
must give exactly the oracle's levels, and exactly what alb_bfs gives, call
after call, although every call reuses the same fixed scratch array inside the
library.

This file is collected last on purpose; it also passes when run on its own.
"""
import numpy as np
import pytest

import oracle
from paper_1911_09135_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_09135_gb300 import alb  # noqa: E402

ALB_ERR_INVALID_ARG, ALB_ERR_DEVICE = 1, 8


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def reference_levels(g, d_off, d_idx, src):
    """Levels from the regular entry point (graph handle, library-owned workspace)."""
    with alb.Graph(g.n, d_off, d_idx, symmetric=g.symmetric) as G:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        G.bfs(src, out)
        G.sync()
        return out.clone()


@pytest.mark.parametrize("which", ["rmat16-directed", "rmat20-sym-max-size"])
def test_noalloc_bfs_equals_oracle_and_alb_bfs_twice(which):
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
        got = host(out).copy()
        assert np.array_equal(got, oracle.bfs(g.n, g.offsets, g.indices, src)), src
        assert torch.equal(out, reference_levels(g, d_off, d_idx, src)), src


def test_noalloc_rejects_graphs_above_the_limit():
    n = alb.ALB_NOALLOC_MAX_VERTICES + 1
    d_off = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(alb.AlbError) as e:
        alb.alb_bfs_noalloc(n, 0, d_off, None, 0, out)
    assert e.value.code == ALB_ERR_INVALID_ARG  # nothing enqueued


@pytest.mark.parametrize("case,offsets,indices,code", [
    ("last offset != m", [0, 1, 2, 3, 3], [1, 2, 3, 0], ALB_ERR_INVALID_ARG),
    ("decreasing offsets", [0, 3, 2, 4, 4], [1, 2, 3, 0], ALB_ERR_INVALID_ARG),
    ("index >= n", [0, 1, 2, 3, 4], [1, 2, 3, 99], ALB_ERR_DEVICE),
])
def test_noalloc_rejects_a_malformed_csr_then_runs_a_good_one(case, offsets, indices, code):
    """The CSR check runs before any round kernel, so a malformed graph is refused without a
    traversal; the next call on a good graph is exact again."""
    n = len(offsets) - 1
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(alb.AlbError) as e:
        alb.alb_bfs_noalloc(n, len(indices), dev(offsets), dev(indices), 0, out)
    assert e.value.code == code, case
    g = gg.from_edges(5, [(0, 1), (1, 2), (2, 3)], None, symmetrize=False, name="path")
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    alb.alb_bfs_noalloc(g.n, g.m, dev(g.offsets), dev(g.indices), 0, out)
    torch.cuda.synchronize()
    assert np.array_equal(host(out), oracle.bfs(g.n, g.offsets, g.indices, 0))
