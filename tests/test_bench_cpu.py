"""Host-side helpers of bench.py: the all-core oracle throughput and the
reporting conventions (no GPU)."""
from __future__ import annotations

import os
import sys

import numpy as np

import graphgen

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_parallel_oracle_throughput():
    off, col = graphgen.kronecker(12, 8, seed=5)
    roots = graphgen.pick_roots(off, 8, seed=6)
    gteps, used, cores = bench.run_oracle_parallel(off, col, roots, 0.0)
    assert gteps > 0 and cores >= 1
    assert len(used) == min(len(roots), cores)
    assert set(used) <= set(int(r) for r in roots)


def test_trimmed_and_harmonic_means():
    x = np.array([1.0, 2.0, 3.0, 4.0, 100.0, 5.0, 6.0, 7.0, 8.0, 0.001])
    # 10 % off each end drops 0.001 and 100
    assert bench.trimmed_mean(x, 0.1) == np.mean([1, 2, 3, 4, 5, 6, 7, 8])
    assert abs(bench.hmean([2.0, 2.0]) - 2.0) < 1e-12
    assert abs(bench.hmean([1.0, 3.0]) - 1.5) < 1e-12
