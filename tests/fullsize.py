"""Helpers of the parity tests at the benchmark sizes: the seeded graphs of
the five workloads (generated once per test session and shared), and the
CPU oracle run over many roots at once on the host cores (the oracle is C
called through ctypes, which releases the GIL)."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import graphgen
import oracle

_CACHE: dict = {}

# (generator, scale, edge factor or average degree, seed) of each workload's graphs
KRON_S22 = ("kronecker", 22, 16, 22)      # single-source headline, 64 roots
KRON_S24 = ("kronecker", 24, 16, 24)      # 64-root batched
ER_S24 = ("erdos_renyi", 24, 32, 25)      # 64-root batched, low skew
SERVE = [("kronecker", s, 16, s) for s in (18, 20, 22, 24)]  # served queries
ROOT_SEED = 3


def graph(spec):
    """The CSR of a workload graph, generated on first use."""
    if spec not in _CACHE:
        kind, scale, k, seed = spec
        gen = graphgen.kronecker if kind == "kronecker" else graphgen.erdos_renyi
        _CACHE[spec] = gen(scale, k, seed=seed)
    return _CACHE[spec]


def oracle_many(off, col, roots, max_levels=4096):
    """oracle.bfs on every root, in parallel on the host cores: a list of
    (dist, parent, info) in the order of roots."""
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda r: oracle.bfs(off, col, int(r), max_levels=max_levels), roots))
