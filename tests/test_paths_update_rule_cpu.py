"""The update rule of the path-count expansion, checked on the CPU against the
oracle under adversarial orderings.

Level L's expansion applies, for each kept entry v -> u of the frontier, in
any order and with each thread reading u's distance either before or after
other threads' stores of the same level:

    h = hops[u]   (the value at level start, or the current one)
    if h == -1 or h == L + 1:  hops[u] = L + 1;  sigma[u] += sigma[v]

and then collects the vertices with hops = L + 1 as the next frontier.
Exact integer counts (Python ints) make the order of the additions
irrelevant, so the model must reproduce the oracle's hops and sigma exactly
whatever the interleaving -- the property the GPU kernel relies on instead
of a compare-and-swap claim.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G


def model(off, col, root, rng, weight=None, lo=0, hi=0):
    n = len(off) - 1
    hops = [-1] * n
    sigma = [0] * n
    hops[root], sigma[root] = 0, 1
    frontier, level = [root], 0
    while frontier:
        entries = [(v, k) for v in frontier for k in range(off[v], off[v + 1])]
        order = rng.permutation(len(entries))
        start = list(hops)                       # what a stale read returns
        for idx in order:
            v, k = entries[idx]
            if weight is not None and not (lo <= weight[k] <= hi):
                continue
            u = int(col[k])
            h = start[u] if rng.random() < 0.5 else hops[u]
            if h == -1 or h == level + 1:
                hops[u] = level + 1
                sigma[u] += sigma[v]
        frontier = [u for u in range(n) if hops[u] == level + 1]
        level += 1
    return np.array(hops), sigma


CASES = [
    ("kron_s7", lambda: graphgen.kronecker(7, 8, 3)),
    ("directed", lambda: G.random_graph(120, 400, 8, undirected=False)),
    ("grid", lambda: G.grid(9, 11)),
    ("duplicates", lambda: (np.array([0, 3, 4, 4], dtype=np.int64),
                            np.array([0, 1, 1, 2], dtype=np.int32))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fire_and_forget_rule_matches_oracle(name, make):
    off, col = make()
    n = len(off) - 1
    rng = np.random.default_rng(17)
    w = rng.integers(0, 4, len(col)).astype(np.int32)
    for r in range(0, n, max(1, n // 6)):
        for weight, lo, hi in ((None, 0, 0), (w, 1, 2)):
            hops, sigma = model(off, col, r, rng, weight, lo, hi)
            eh, es, _ = oracle.bfs_paths(off, col, r, weight, lo, hi)
            assert np.array_equal(hops, eh)
            assert [float(x) for x in sigma] == es.tolist()
