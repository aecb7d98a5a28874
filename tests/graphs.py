"""Hand-built test graphs (fixtures only; no traversal arithmetic)."""
from paper_1911_09135_gb300 import graphgen as gg


def path(n, weighted=True):
    e = [(i, i + 1) for i in range(n - 1)]
    return gg.from_edges(n, e, [1 + (i % 7) for i in range(len(e))] if weighted else None,
                         symmetrize=True, name=f"path{n}")


def star(n, weighted=True):
    e = [(0, i) for i in range(1, n)]
    return gg.from_edges(n, e, [1 + (i % 5) for i in range(len(e))] if weighted else None,
                         symmetrize=True, name=f"star{n}")


def complete(n, weighted=True):
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return gg.from_edges(n, e, [1 + ((i * 3 + j) % 9) for i, j in e] if weighted else None,
                         symmetrize=True, name=f"complete{n}")


def cycle(n, weighted=True):
    e = [(i, (i + 1) % n) for i in range(n)]
    return gg.from_edges(n, e, [2] * len(e) if weighted else None, symmetrize=True,
                         name=f"cycle{n}")


def two_components(weighted=True):
    e = [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 6)]
    return gg.from_edges(8, e, [3, 1, 4, 1, 5, 9] if weighted else None, symmetrize=True,
                         name="two-components+isolated")


def messy_input(weighted=True):
    """Self-loops and duplicate entries in the raw edge list (removed by from_edges)."""
    e = [(0, 0), (0, 1), (0, 1), (1, 2), (2, 2), (2, 3), (3, 1), (1, 2)]
    return gg.from_edges(5, e, [1, 2, 2, 3, 4, 5, 6, 3] if weighted else None, symmetrize=True,
                         name="selfloop-dup")


def empty(n=1):
    return gg.from_edges(n, [], [], symmetrize=True, name=f"empty{n}")


def directed_cycle_tail():
    e = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (5, 4)]
    return gg.from_edges(6, e, [1, 2, 3, 4, 5, 6], symmetrize=False, name="directed")


def all_small():
    return [path(9), star(12), complete(6), cycle(7), two_components(), messy_input(), empty(1),
            empty(4)]
