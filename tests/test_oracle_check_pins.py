"""Pins for the certificate checker (oracle.check_bfs, bfs_check.c).

The checker claims: with no parent array it accepts a distance array
exactly when it equals the hop distances from the root (the result of
Algorithm 1, Section "Preliminaries"), and with a parent array it accepts
exactly when, in addition, every reached vertex but the root has a parent
joined to it by a CSR entry and one level closer (root: itself; unreached:
-1).  Both claims are tested by exhaustive enumeration on tiny graphs --
every array of values in [-2, n) or [-1, n) -- against Floyd-Warshall distances and
the definition of a valid parent written out here; then each planted
mistake in a copy of the checker's source must break one of those pins.
Larger graphs: the oracle's own output is accepted with any thread count,
perturbations are rejected, and the verdicts agree with check_tree.
"""
from __future__ import annotations

import itertools
import os
import subprocess

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G
from tests.test_oracle_pins import floyd_warshall


def _csr_from_entries(n, entries):
    rows = [[] for _ in range(n)]
    for a, b in entries:
        rows[a].append(b)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([b for r in rows for b in r], dtype=np.int32)
    return off, col


# tiny graphs: directed and undirected, with duplicates, self-loops, isolated
# vertices and vertices that reach nothing
TINY = [
    ("path4", lambda: G.path(4), 0),
    ("directed_chain_dup", lambda: _csr_from_entries(5, [(0, 1), (0, 1), (1, 2), (2, 3), (3, 3),
                                                         (0, 2)]), 0),
    ("directed_fork", lambda: _csr_from_entries(5, [(1, 0), (1, 2), (2, 4), (0, 4), (4, 1)]), 1),
    ("cycle5", lambda: G.cycle(5), 2),
    ("isolated", lambda: _csr_from_entries(5, [(0, 1), (1, 0), (1, 2), (2, 1)]), 2),
    ("star_in", lambda: _csr_from_entries(5, [(1, 0), (2, 0), (3, 0), (4, 0), (0, 0)]), 0),
    ("root_last", lambda: _csr_from_entries(5, [(4, 0), (0, 1), (4, 2), (2, 3)]), 4),
]


def _valid_parent(off, col, root, dist, parent):
    """The definition: parent[root] = root; unreached -> -1; a reached v !=
    root has parent p with a CSR entry p -> v and dist[p] = dist[v] - 1."""
    n = len(off) - 1
    if parent[root] != root:
        return False
    for v in range(n):
        if v == root:
            continue
        p = parent[v]
        if dist[v] < 0:
            if p != -1:
                return False
            continue
        if not (0 <= p < n) or dist[p] != dist[v] - 1:
            return False
        if v not in set(col[off[p]:off[p + 1]].tolist()):
            return False
    return True


def _accepts(off, col, root, dist, parent=None, lib=None, nthreads=2):
    return oracle.check_bfs(off, col, root, dist, parent, nthreads=nthreads, lib=lib)["ok"]


def _exhaustive_dist(off, col, root, lib=None):
    """Every dist array in [-2, n)^n (-2: a value no result may hold):
    accepted exactly for the true one."""
    n = len(off) - 1
    truth = floyd_warshall(off, col)[root]
    accepted = []
    for cand in itertools.product(range(-2, n), repeat=n):
        d = np.array(cand, dtype=np.int32)
        if _accepts(off, col, root, d, lib=lib):
            accepted.append(cand)
    return accepted == [tuple(int(x) for x in truth)]


def _exhaustive_parent(off, col, root, lib=None):
    """Every parent array in [-1, n)^n with the true distances: accepted
    exactly when the definition holds."""
    n = len(off) - 1
    truth = floyd_warshall(off, col)[root].astype(np.int32)
    for cand in itertools.product(range(-1, n), repeat=n):
        p = np.array(cand, dtype=np.int32)
        if _accepts(off, col, root, truth, p, lib=lib) != _valid_parent(off, col, root, truth, p):
            return False
    return True


@pytest.mark.parametrize("name,make,root", TINY, ids=[t[0] for t in TINY])
def test_checker_accepts_exactly_the_true_distances(name, make, root):
    off, col = make()
    assert _exhaustive_dist(off, col, root)


@pytest.mark.parametrize("name,make,root", TINY[:4], ids=[t[0] for t in TINY[:4]])
def test_checker_parent_rules_match_the_definition(name, make, root):
    off, col = make()
    assert _exhaustive_parent(off, col, root)


def test_checker_agrees_with_oracle_and_check_tree_kronecker():
    off, col = graphgen.kronecker(13, 8, seed=5)
    roots = graphgen.pick_roots(off, 4, seed=9)
    rng = np.random.default_rng(1)
    for r in roots:
        r = int(r)
        d, p, info = oracle.bfs(off, col, r)
        for nt in (1, 3, 8):
            res = oracle.check_bfs(off, col, r, d, p, nthreads=nt)
            assert res["ok"], res
            assert res["edges_scanned"] == info["edges_scanned"]
            assert res["levels"] == info["levels"]
            assert res["reached"] == info["reached"]
        # int8 rows are checked through their int32 values
        assert oracle.check_bfs(off, col, r, d.astype(np.int8))["ok"]
        for _ in range(6):
            d2, p2 = d.copy(), p.copy()
            v = int(rng.choice(np.nonzero(d > 0)[0]))
            kind = rng.integers(0, 4)
            if kind == 0:
                d2[v] += 1
            elif kind == 1:
                d2[v] -= 1
            elif kind == 2:
                d2[v] = -1
            else:
                p2[v] = r if d[v] != 1 else int(np.nonzero(d == 2)[0][0])
            res = oracle.check_bfs(off, col, r, d2, p2)
            assert not res["ok"]
            assert oracle.check_tree(off, col, r, d2, p2) != []


MUTATIONS = [
    ("no_reach_gap", "t->bad[BAD_REACH_GAP] += 1;", "t->bad[BAD_REACH_GAP] += 0;"),
    ("no_level_skip", "t->bad[BAD_LEVEL_SKIP] += 1;", "t->bad[BAD_LEVEL_SKIP] += 0;"),
    ("skip_tolerance_two", "} else if (dv > du + 1) {", "} else if (dv > du + 2) {"),
    ("no_witness_check", "if (!t->witness[x]) t->bad[BAD_NO_WITNESS] += 1;",
     "if (!t->witness[x]) t->bad[BAD_NO_WITNESS] += 0;"),
    ("witness_same_level", "} else if (dv == du + 1) {", "} else if (dv == du) {"),
    ("no_range_check", "t->bad[BAD_RANGE] += 1;", "t->bad[BAD_RANGE] += 0;"),
    ("no_root_check", "if (dist[root] != 0) bad[BAD_ROOT_DIST] += 1;",
     "if (dist[root] != 0) bad[BAD_ROOT_DIST] += 0;"),
    ("drop_last_entry", "e < t->off[u + 1]; ++e", "e < t->off[u + 1] - 1; ++e"),
    ("last_range_short", "            v = n;\n", "            v = n - 1;\n"),
    ("no_parent_check", "if (t->parent && !t->entry[x])", "if (0)"),
    ("parent_mark_any", "if (t->parent && t->parent[v] == (int32_t)u)",
     "if (t->parent && t->parent[v] != -1)"),
    ("no_root_parent", "bad[BAD_ROOT_PARENT] += 1;", "bad[BAD_ROOT_PARENT] += 0;"),
    ("no_unreached_parent", "if (t->parent && t->parent[x] != -1) t->bad[BAD_UNREACHED_PARENT] += 1;",
     "if (t->parent && t->parent[x] != -1) t->bad[BAD_UNREACHED_PARENT] += 0;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_checker_mistakes(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bfs_check.c")).read()
    assert old in src
    mutated = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(mutated)
    so = str(tmp_path / f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-pthread", "-shared", "-fPIC", "-o", so, str(path)])
    lib = oracle.load_check(so)
    caught = False
    for _, make, root in TINY:
        off, col = make()
        if not _exhaustive_dist(off, col, root, lib=lib) or \
                not _exhaustive_parent(off, col, root, lib=lib):
            caught = True
            break
    assert caught, f"mutation {name} not caught by any pin"
