"""Generator pins: edge counts, R-MAT quadrant frequencies, cleanup
properties, permutation, determinism and root picking."""
from __future__ import annotations

import numpy as np

import graphgen


def test_rmat_generated_edge_count_config_scale16():
    src, dst = graphgen.rmat_edges_raw(16, 8 << 16, seed=1)
    assert len(src) == 524_288 and len(dst) == 524_288
    assert src.min() >= 0 and src.max() < 1 << 16


def test_rmat_quadrant_frequencies():
    scale, m = 10, 200_000
    src, dst = graphgen.rmat_edges_raw(scale, m, seed=7, permute=False)
    a, b, c = graphgen.RMAT_A, graphgen.RMAT_B, graphgen.RMAT_C
    probs = np.array([a, b, c, 1 - a - b - c])
    for bit in (0, scale - 1):
        sb = (src >> bit) & 1
        db = (dst >> bit) & 1
        freq = np.bincount(sb * 2 + db, minlength=4) / m
        sigma = np.sqrt(probs * (1 - probs) / m)
        assert np.all(np.abs(freq - probs) < 5 * sigma), (bit, freq)


def test_permutation_is_a_relabelling():
    s1, d1 = graphgen.rmat_edges_raw(9, 5000, seed=3, permute=False)
    s2, d2 = graphgen.rmat_edges_raw(9, 5000, seed=3, permute=True)
    # same edge list under one bijection
    mapping = {}
    for x, y in zip(np.concatenate([s1, d1]), np.concatenate([s2, d2])):
        assert mapping.setdefault(int(x), int(y)) == int(y)
    assert len(set(mapping.values())) == len(mapping)


def test_cleanup_properties():
    for off, col in (graphgen.kronecker(12, 8, 5), graphgen.erdos_renyi(11, 8, 5),
                     graphgen.kronecker(11, 16, 6)):
        n = len(off) - 1
        assert off[0] == 0 and off[-1] == len(col)
        assert np.all(np.diff(off) >= 0)
        src = np.repeat(np.arange(n), np.diff(off))
        assert np.all(src != col), "self-loop"
        key = src * n + col
        assert np.all(np.diff(key) > 0), "rows not sorted/deduplicated"
        rev = np.sort(col.astype(np.int64) * n + src)
        assert np.array_equal(rev, key), "not symmetric"


def test_determinism_and_seed_sensitivity():
    o1, c1 = graphgen.kronecker(10, 8, 42)
    o2, c2 = graphgen.kronecker(10, 8, 42)
    o3, c3 = graphgen.kronecker(10, 8, 43)
    assert np.array_equal(o1, o2) and np.array_equal(c1, c2)
    assert not (len(c1) == len(c3) and np.array_equal(c1, c3))


def test_er_mean_degree():
    off, col = graphgen.erdos_renyi(14, 32, 9)
    n = len(off) - 1
    assert 31.0 < len(col) / n <= 32.0


def test_pick_roots():
    off, col = graphgen.kronecker(12, 8, 1)
    roots = graphgen.pick_roots(off, 64, 5)
    deg = np.diff(off)
    assert len(set(roots.tolist())) == 64
    assert np.all(deg[roots] >= 1)
    assert np.array_equal(roots, graphgen.pick_roots(off, 64, 5))
