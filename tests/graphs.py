"""Small hand-built graphs with closed-form BFS distances, as CSR.

Each builder returns (off int64[n+1], col int32[m]) with rows sorted.
"""
from __future__ import annotations

import numpy as np


def from_edges(n, src, dst, undirected=True):
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if undirected:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    keep = src != dst
    src, dst = src[keep], dst[keep]
    key = np.unique(src * n + dst)
    src, dst = key // n, key % n
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    np.cumsum(off, out=off)
    return off, dst.astype(np.int32)


def path(n):
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1)


def directed_path(n):
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, undirected=False)


def cycle(n):
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n)


def star(n):
    leaves = np.arange(1, n)
    return from_edges(n, np.zeros(n - 1, dtype=np.int64), leaves)


def complete(n):
    a, b = np.triu_indices(n, 1)
    return from_edges(n, a, b)


def hypercube(d):
    n = 1 << d
    src, dst = [], []
    for bit in range(d):
        v = np.arange(n)
        src.append(v)
        dst.append(v ^ (1 << bit))
    return from_edges(n, np.concatenate(src), np.concatenate(dst))


def grid(a, b):
    idx = np.arange(a * b).reshape(a, b)
    src = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    dst = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(a * b, src, dst)


def binary_tree(n):
    child = np.arange(1, n)
    return from_edges(n, (child - 1) // 2, child)


def disjoint_union(g1, g2):
    off1, col1 = g1
    off2, col2 = g2
    n1 = len(off1) - 1
    off = np.concatenate([off1, off2[1:] + off1[-1]])
    col = np.concatenate([col1, col2 + n1]).astype(np.int32)
    return off, col


def random_graph(n, m, seed, undirected=True):
    rng = np.random.default_rng(seed)
    return from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m), undirected)


def tree_distance(n, r):
    """Closed form in a heap-indexed complete binary tree: depth(i) + depth(r)
    - 2 depth(lca(i, r))."""
    def depth(x):
        return int(np.floor(np.log2(x + 1)))

    out = np.empty(n, dtype=np.int64)
    for i in range(n):
        a, b = i, r
        da, db = depth(a), depth(b)
        d0a, d0b = da, db
        while da > db:
            a = (a - 1) // 2
            da -= 1
        while db > da:
            b = (b - 1) // 2
            db -= 1
        while a != b:
            a = (a - 1) // 2
            b = (b - 1) // 2
            da -= 1
        out[i] = d0a + d0b - 2 * da
    return out
