"""Pins for the CPU oracle: it is checked against things other than itself.

* Floyd-Warshall brute force (integer min-plus closure) on random directed and
  undirected graphs, and on small Kronecker graphs, every root.
* Closed-form distances: path, directed path, cycle, star, complete graph,
  hypercube (popcount(i xor r)), 2-D grid (Manhattan), complete binary tree
  (depth sum minus twice the LCA depth), disjoint union (-1 across parts),
  single vertex and degree-0 root.
* scipy's breadth-first search (csgraph.shortest_path, unweighted) on larger
  Kronecker graphs.
* Level structure (Section "Preliminaries": level k = vertices at distance
  k): per-level counts equal the distance histogram and sum to the reached
  count; reached set equals the root's connected component from scipy's
  union-find-based connected_components.
* Graph500-style invariants of the oracle's own parents.
* Mutation checks: each planted mistake in a copy of the oracle source fails
  at least one of these pins.
"""
from __future__ import annotations

import os
import re
import subprocess

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G


def floyd_warshall(off, col):
    n = len(off) - 1
    inf = 1 << 40
    d = np.full((n, n), inf, dtype=np.int64)
    np.fill_diagonal(d, 0)
    src = np.repeat(np.arange(n), np.diff(off))
    d[src, col] = np.minimum(d[src, col], 1)
    for k in range(n):
        np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :], out=d)
    d[d >= inf] = -1
    return d


def all_roots_equal_fw(off, col, lib=None, roots=None):
    fw = floyd_warshall(off, col)
    n = len(off) - 1
    for r in (range(n) if roots is None else roots):
        dist, _, _ = oracle.bfs(off, col, r, lib=lib)
        if not np.array_equal(dist, fw[r]):
            return False
    return True


FW_CASES = [
    ("undirected_sparse", lambda: G.random_graph(60, 80, 1)),
    ("undirected_dense", lambda: G.random_graph(40, 400, 2)),
    ("directed_sparse", lambda: G.random_graph(70, 140, 3, undirected=False)),
    ("directed_isolated", lambda: G.random_graph(90, 60, 4, undirected=False)),
    ("kron_s6", lambda: graphgen.kronecker(6, 4, 11)),
    ("kron_s8", lambda: graphgen.kronecker(8, 8, 12)),
    ("er_s7", lambda: graphgen.erdos_renyi(7, 4, 13)),
]


@pytest.mark.parametrize("name,make", FW_CASES, ids=[c[0] for c in FW_CASES])
def test_oracle_matches_floyd_warshall_every_root(name, make):
    off, col = make()
    assert all_roots_equal_fw(off, col)


def test_oracle_matches_floyd_warshall_scale10():
    off, col = graphgen.kronecker(10, 4, 21)
    rng = np.random.default_rng(0)
    roots = rng.choice(len(off) - 1, 48, replace=False)
    assert all_roots_equal_fw(off, col, roots=roots)


def _closed_form_cases():
    cases = []
    n = 23
    off, col = G.path(n)
    for r in (0, 7, n - 1):
        cases.append((f"path_r{r}", off, col, r, np.abs(np.arange(n) - r)))
    off, col = G.directed_path(n)
    for r in (0, 9):
        exp = np.where(np.arange(n) >= r, np.arange(n) - r, -1)
        cases.append((f"dpath_r{r}", off, col, r, exp))
    off, col = G.cycle(n)
    for r in (0, 5):
        k = np.abs(np.arange(n) - r)
        cases.append((f"cycle_r{r}", off, col, r, np.minimum(k, n - k)))
    off, col = G.star(17)
    cases.append(("star_center", off, col, 0, np.r_[0, np.ones(16, dtype=np.int64)]))
    exp = np.full(17, 2)
    exp[0], exp[5] = 1, 0
    cases.append(("star_leaf", off, col, 5, exp))
    off, col = G.complete(12)
    exp = np.ones(12, dtype=np.int64)
    exp[3] = 0
    cases.append(("complete", off, col, 3, exp))
    off, col = G.hypercube(6)
    for r in (0, 45):
        exp = np.array([bin(i ^ r).count("1") for i in range(64)])
        cases.append((f"hypercube_r{r}", off, col, r, exp))
    a, b = 7, 9
    off, col = G.grid(a, b)
    for r in (0, 31):
        ii, jj = np.divmod(np.arange(a * b), b)
        ri, rj = divmod(r, b)
        cases.append((f"grid_r{r}", off, col, r, np.abs(ii - ri) + np.abs(jj - rj)))
    off, col = G.binary_tree(40)
    for r in (0, 17, 39):
        cases.append((f"tree_r{r}", off, col, r, G.tree_distance(40, r)))
    off, col = G.disjoint_union(G.path(5), G.cycle(6))
    cases.append(("union_left", off, col, 2, np.r_[2, 1, 0, 1, 2, -np.ones(6, dtype=np.int64)]))
    cases.append(("union_right", off, col, 5, np.r_[-np.ones(5, dtype=np.int64), 0, 1, 2, 3, 2, 1]))
    off = np.zeros(2, dtype=np.int64)
    cases.append(("single_vertex", off, np.zeros(0, dtype=np.int32), 0, np.array([0])))
    off, col = G.disjoint_union((np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32)), G.cycle(4))
    cases.append(("deg0_root", off, col, 0, np.array([0, -1, -1, -1, -1])))
    return cases


CLOSED = _closed_form_cases()


@pytest.mark.parametrize("case", CLOSED, ids=[c[0] for c in CLOSED])
def test_oracle_closed_forms(case):
    _, off, col, r, expected = case
    dist, parent, info = oracle.bfs(off, col, r)
    assert np.array_equal(dist, np.asarray(expected, dtype=np.int32))
    assert oracle.check_tree(off, col, r, dist, parent, undirected=not case[0].startswith("dpath")) == []
    assert info["reached"] == int(np.count_nonzero(np.asarray(expected) >= 0))


def test_oracle_matches_scipy_bfs_kronecker():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    off, col = graphgen.kronecker(13, 8, 5)
    n = len(off) - 1
    a = sp.csr_matrix((np.ones(len(col)), col, off), shape=(n, n))
    roots = graphgen.pick_roots(off, 6, 99)
    ref = csgraph.shortest_path(a, method="D", unweighted=True, indices=roots)
    ref = np.where(np.isinf(ref), -1, ref).astype(np.int64)
    for i, r in enumerate(roots):
        dist, _, _ = oracle.bfs(off, col, r)
        assert np.array_equal(dist, ref[i])


def test_oracle_levels_and_components():
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    sp = pytest.importorskip("scipy.sparse")
    off, col = graphgen.kronecker(12, 8, 6)
    n = len(off) - 1
    ncomp, labels = csgraph.connected_components(
        sp.csr_matrix((np.ones(len(col)), col, off), shape=(n, n)), directed=False)
    assert ncomp > 1  # Kronecker graphs have isolated vertices
    for r in graphgen.pick_roots(off, 5, 3):
        dist, parent, info = oracle.bfs(off, col, r)
        reached = dist >= 0
        assert np.array_equal(reached, labels == labels[r])
        hist = np.bincount(dist[reached], minlength=info["levels"])
        assert np.array_equal(hist, info["level_sizes"])
        assert info["level_sizes"].sum() == info["reached"]
        deg = np.diff(off)
        assert info["edges_scanned"] == int(deg[reached].sum())
        assert oracle.check_tree(off, col, r, dist, parent) == []


def test_oracle_multi_is_rowwise():
    off, col = graphgen.kronecker(9, 8, 8)
    roots = np.array([3, 3, 100, 511, 0])
    dist, scanned = oracle.bfs_multi(off, col, roots)
    for i, r in enumerate(roots):
        d, _, info = oracle.bfs(off, col, r)
        assert np.array_equal(dist[i], d)
        assert scanned[i] == info["edges_scanned"]


def test_oracle_rejects_bad_root():
    off, col = G.path(4)
    with pytest.raises(ValueError):
        oracle.bfs(off, col, 4)


def test_check_tree_catches_bad_parents():
    off, col = graphgen.kronecker(9, 8, 8)
    r = int(graphgen.pick_roots(off, 1, 1)[0])
    dist, parent, _ = oracle.bfs(off, col, r)
    assert oracle.check_tree(off, col, r, dist, parent) == []
    v = int(np.nonzero(dist == 2)[0][0])
    bad = parent.copy()
    bad[v] = r  # root is not adjacent to a level-2 vertex
    assert oracle.check_tree(off, col, r, dist, bad) != []
    bad = parent.copy()
    bad[r] = -1
    assert oracle.check_tree(off, col, r, dist, bad) != []
    d2 = dist.copy()
    d2[v] += 1
    assert oracle.check_tree(off, col, r, d2, parent) != []


MUTATIONS = [
    ("dist_plus_two", "dist[u] = dv + 1;", "dist[u] = dv + 2;"),
    ("revisit_root", "if (dist[u] == -1)", "if (dist[u] <= 0)"),
    ("drop_last_neighbour", "e < off[v + 1]; ++e", "e < off[v + 1] - 1; ++e"),
    ("root_dist_one", "dist[root] = 0;", "dist[root] = 1;"),
    ("lifo_queue", "int32_t v = queue[head++];", "int32_t v = queue[--tail]; ++head; tail += 0;"),
    ("init_zero", "dist[v] = -1;", "dist[v] = 0;"),
    ("skip_first_neighbour", "int64_t e = off[v];", "int64_t e = off[v] + 1;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_oracle_mistakes(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bfs_oracle.c")).read()
    assert old in src
    if name == "lifo_queue":
        # stack discipline: pop from the tail instead of the head
        mutated = src.replace("while (head < tail) {\n        int32_t v = queue[head++];",
                              "while (tail > 0) {\n        int32_t v = queue[--tail];")
        assert mutated != src
    else:
        mutated = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(mutated)
    so = str(tmp_path / f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", so, str(path)])
    lib = oracle.load(so)
    caught = False
    for _, make in FW_CASES[:4]:
        off, col = make()
        try:
            if not all_roots_equal_fw(off, col, lib=lib):
                caught = True
                break
        except Exception:
            caught = True
            break
    if not caught:
        for case in CLOSED:
            _, off, col, r, expected = case
            d, _, _ = oracle.bfs(off, col, r, lib=lib)
            if not np.array_equal(d, np.asarray(expected)):
                caught = True
                break
    assert caught, f"mutation {name} not caught by any pin"
