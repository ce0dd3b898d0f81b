"""Pins for the oracle's shortest-path counts (``oracle.bfs_paths``), checked
against definitions that share nothing with a breadth-first search:

* Walk counts from adjacency-matrix powers: the number of walks of length k
  from r to v is (A^k)[r, v] (A counts kept entries, so a duplicated entry
  counts twice); the smallest k with a non-zero count is the distance, and
  a walk of that length repeats no vertex, so the count is the number of
  shortest paths.  Exact Python integers, every root of small random
  directed and undirected graphs and small Kronecker graphs, with and
  without a weight filter.
* Closed forms: 2-D grid from a corner (binomial coefficients), hypercube
  (popcount(x)!), complete graph, even cycle (2 paths to the antipode),
  complete bipartite graph, star, path.
* Weight filters with known reach: a grid whose horizontal entries weigh 1
  and vertical ones 2; an empty filter range; scipy's unweighted shortest
  paths on the filtered subgraph of a scale-10 Kronecker graph.
* Mutation checks: each planted mistake in a copy of the oracle source
  fails at least one of these pins.
"""
from __future__ import annotations

import math
import os
import subprocess

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G


def walk_counts(off, col, root, keep=None):
    n = len(off) - 1
    a = np.zeros((n, n), dtype=object)
    src = np.repeat(np.arange(n), np.diff(off))
    for i, (s, d) in enumerate(zip(src, col)):
        if keep is None or keep[i]:
            a[s, d] += 1
    hops = np.full(n, -1, dtype=np.int64)
    sigma = np.zeros(n, dtype=object)
    row = np.zeros(n, dtype=object)
    row[root] = 1
    for k in range(n):
        new = (hops < 0) & (row > 0)
        hops[new] = k
        sigma[new] = row[new]
        row = row.dot(a)
    return hops, sigma


def matches_walks(off, col, roots, weight=None, lo=0, hi=0, lib=None):
    keep = None if weight is None else (weight >= lo) & (weight <= hi)
    for r in roots:
        hops, sigma, _ = oracle.bfs_paths(off, col, r, weight, lo, hi, lib=lib)
        eh, es = walk_counts(off, col, r, keep)
        if not np.array_equal(hops, eh):
            return False
        if any(float(x) != float(y) for x, y in zip(sigma, es)):
            return False
    return True


WALK_CASES = [
    ("undirected_sparse", lambda: G.random_graph(24, 30, 1)),
    ("undirected_dense", lambda: G.random_graph(20, 90, 2)),
    ("directed", lambda: G.random_graph(26, 70, 3, undirected=False)),
    ("directed_isolated", lambda: G.random_graph(30, 25, 4, undirected=False)),
    ("kron_s5", lambda: graphgen.kronecker(5, 4, 11)),
]


def weights_for(col, seed):
    return np.random.default_rng(seed).integers(0, 4, len(col)).astype(np.int32)


@pytest.mark.parametrize("name,make", WALK_CASES, ids=[c[0] for c in WALK_CASES])
def test_paths_match_walk_counts(name, make):
    off, col = make()
    n = len(off) - 1
    assert matches_walks(off, col, range(n))
    w = weights_for(col, 7)
    assert matches_walks(off, col, range(n), w, 1, 2)
    assert matches_walks(off, col, range(0, n, 3), w, 3, 3)


def test_paths_duplicate_entries_count_twice():
    # 0 -> 1 stored twice, 1 -> 2, 0 -> 2 absent: two shortest paths to 2
    off = np.array([0, 2, 3, 3], dtype=np.int64)
    col = np.array([1, 1, 2], dtype=np.int32)
    hops, sigma, info = oracle.bfs_paths(off, col, 0)
    assert hops.tolist() == [0, 1, 2]
    assert sigma.tolist() == [1.0, 2.0, 2.0]
    assert info["edges_scanned"] == 3
    assert matches_walks(off, col, [0, 1, 2])


def bipartite(a, b):
    left = np.repeat(np.arange(a), b)
    right = np.tile(np.arange(a, a + b), a)
    return G.from_edges(a + b, left, right)


def test_paths_closed_forms():
    rows, cols = 5, 7
    off, col = G.grid(rows, cols)
    hops, sigma, _ = oracle.bfs_paths(off, col, 0)
    for i in range(rows):
        for j in range(cols):
            assert hops[i * cols + j] == i + j
            assert sigma[i * cols + j] == math.comb(i + j, i)
    d = 7
    off, col = G.hypercube(d)
    hops, sigma, _ = oracle.bfs_paths(off, col, 0)
    for x in range(1 << d):
        assert hops[x] == bin(x).count("1")
        assert sigma[x] == math.factorial(bin(x).count("1"))
    off, col = G.complete(9)
    hops, sigma, _ = oracle.bfs_paths(off, col, 4)
    assert hops.tolist() == [1, 1, 1, 1, 0, 1, 1, 1, 1]
    assert sigma.tolist() == [1.0] * 9
    off, col = G.cycle(10)
    hops, sigma, _ = oracle.bfs_paths(off, col, 0)
    assert hops.tolist() == [0, 1, 2, 3, 4, 5, 4, 3, 2, 1]
    assert sigma.tolist() == [1, 1, 1, 1, 1, 2, 1, 1, 1, 1]
    off, col = bipartite(3, 4)
    hops, sigma, _ = oracle.bfs_paths(off, col, 0)
    assert hops.tolist() == [0, 2, 2, 1, 1, 1, 1]
    assert sigma.tolist() == [1, 4, 4, 1, 1, 1, 1]
    off, col = G.star(6)
    hops, sigma, _ = oracle.bfs_paths(off, col, 3)
    assert hops.tolist() == [1, 2, 2, 0, 2, 2]
    assert sigma.tolist() == [1, 1, 1, 1, 1, 1]
    off, col = G.path(6)
    hops, sigma, _ = oracle.bfs_paths(off, col, 2)
    assert hops.tolist() == [2, 1, 0, 1, 2, 3]
    assert sigma.tolist() == [1] * 6
    off, col = G.disjoint_union(G.path(3), G.cycle(4))
    hops, sigma, _ = oracle.bfs_paths(off, col, 0)
    assert hops.tolist() == [0, 1, 2, -1, -1, -1, -1]
    assert sigma.tolist() == [1, 1, 1, 0, 0, 0, 0]


def grid_weights(off, col, cols):
    """Horizontal entries (same row) weigh 1, vertical ones 2."""
    n = len(off) - 1
    src = np.repeat(np.arange(n), np.diff(off))
    return np.where(src // cols == col // cols, 1, 2).astype(np.int32)


def test_paths_weight_filter_on_grid():
    rows, cols = 4, 6
    off, col = G.grid(rows, cols)
    w = grid_weights(off, col, cols)
    full_h, full_s, _ = oracle.bfs_paths(off, col, 0)
    hops, sigma, _ = oracle.bfs_paths(off, col, 0, w, 1, 2)
    assert np.array_equal(hops, full_h) and np.array_equal(sigma, full_s)
    hops, sigma, info = oracle.bfs_paths(off, col, 0, w, 1, 1)      # row 0 only
    expect = np.full(rows * cols, -1)
    expect[:cols] = np.arange(cols)
    assert np.array_equal(hops, expect)
    assert np.array_equal(sigma, (expect >= 0).astype(float))
    assert info["edges_scanned"] == int(np.diff(off)[:cols].sum())
    hops, sigma, _ = oracle.bfs_paths(off, col, 0, w, 2, 2)         # column 0 only
    expect = np.full(rows * cols, -1)
    expect[::cols] = np.arange(rows)
    assert np.array_equal(hops, expect)
    hops, sigma, info = oracle.bfs_paths(off, col, 7, w, 3, 1)      # empty range
    assert hops.tolist() == [0 if v == 7 else -1 for v in range(rows * cols)]
    assert sigma.sum() == 1.0 and info["levels"] == 1


def test_paths_filtered_hops_match_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    off, col = graphgen.kronecker(10, 8, 5)
    n = len(off) - 1
    w = weights_for(col, 9)
    keep = (w >= 0) & (w <= 1)
    src = np.repeat(np.arange(n), np.diff(off))
    a = sp.csr_matrix((np.ones(int(keep.sum())), (src[keep], col[keep])), shape=(n, n))
    for r in [0, 17, 333, 1000]:
        d = csgraph.shortest_path(a, method="D", unweighted=True, directed=True, indices=r)
        expect = np.where(np.isinf(d), -1, d).astype(np.int64)
        hops, sigma, _ = oracle.bfs_paths(off, col, r, w, 0, 1)
        assert np.array_equal(hops, expect)
        assert np.all((sigma > 0) == (hops >= 0))


PATH_MUTATIONS = [
    ("first_contribution_only", "if (hops[b] == ha + 1) sigma[b] += sigma[a];",
     "if (hops[b] == ha + 1 && sigma[b] == 0.0) sigma[b] += sigma[a];"),
    ("filter_drops_low_bound", "weight[k] < lo ||", "weight[k] <= lo ||"),
    ("root_count_two", "sigma[root] = 1.0;", "sigma[root] = 2.0;"),
    ("same_level_entries", "if (hops[b] == ha + 1) sigma", "if (hops[b] >= ha) sigma"),
    ("hops_plus_two", "hops[b] = ha + 1;", "hops[b] = ha + 2;"),
    ("skip_last_entry", "k < off[a + 1]; ++k", "k < off[a + 1] - 1; ++k"),
    ("filter_ignored", "if (weight && (", "if (0 && ("),
]


def pins_hold(lib):
    try:
        for _, make in WALK_CASES[:3]:
            off, col = make()
            n = len(off) - 1
            if not matches_walks(off, col, range(0, n, 2), lib=lib):
                return False
            if not matches_walks(off, col, range(0, n, 2), weights_for(col, 7), 1, 2, lib=lib):
                return False
        off, col = G.grid(4, 6)
        w = grid_weights(off, col, 6)
        hops, _, _ = oracle.bfs_paths(off, col, 0, w, 1, 1, lib=lib)
        if hops[:6].tolist() != list(range(6)) or np.any(hops[6:] != -1):
            return False
    except Exception:
        return False
    return True


def test_paths_pins_hold_for_the_oracle():
    assert pins_hold(oracle.load())


@pytest.mark.parametrize("name,old,new", PATH_MUTATIONS, ids=[m[0] for m in PATH_MUTATIONS])
def test_paths_pins_catch_planted_mistakes(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bfs_oracle.c")).read()
    assert src.count(old) == 1
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", so, str(path)])
    assert not pins_hold(oracle.load(so)), f"mutation {name} not caught"
