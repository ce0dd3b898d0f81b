"""Autotuner: picks bin thresholds / chunk sizes / CTAs per SM by timing,
applies them, caches by graph fingerprint; results stay bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


def test_autotune_applies_and_caches(tmp_path):
    ctx = bfs.Context(0)
    off, col = graphgen.kronecker(15, 16, seed=4)
    n = len(off) - 1
    roots = graphgen.pick_roots(off, 4, seed=5)
    g = bfs.Graph(ctx, off, col)
    cache = str(tmp_path / "tune.jsonl")
    r1 = g.autotune(roots, cache_path=cache)
    assert r1["from_cache"] == 0 and r1["trials"] > 5 and r1["best_ms"] > 0
    info = g.info()
    assert (info["t_small"], info["t_large"], info["chunk_warp"], info["chunk_cta"]) == \
        (r1["t_small"], r1["t_large"], r1["chunk_warp"], r1["chunk_cta"])
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:
        g.run(int(r), d, p)
        g.sync()
        ref, _, _ = oracle.bfs(off, col, int(r))
        assert np.array_equal(d.cpu().numpy(), ref)
        assert oracle.check_tree(off, col, int(r), d.cpu().numpy(), p.cpu().numpy()) == []
    # same graph uploaded again: the cache answers without timing
    g2 = bfs.Graph(ctx, off, col)
    r2 = g2.autotune(roots, cache_path=cache)
    assert r2["from_cache"] == 1 and r2["trials"] == 0
    assert r2["fingerprint"] == r1["fingerprint"]
    assert (r2["t_small"], r2["t_large"], r2["chunk_warp"], r2["chunk_cta"], r2["ctas_per_sm"]) == \
        (r1["t_small"], r1["t_large"], r1["chunk_warp"], r1["chunk_cta"], r1["ctas_per_sm"])
    # batched tuning is a separate cache entry
    rb = g2.autotune(roots, batched=True, cache_path=cache)
    assert rb["from_cache"] == 0
    bd = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    g2.run_batch(roots, bd)
    g2.batch_sync()
    ref, _ = oracle.bfs_multi(off, col, roots)
    assert np.array_equal(bd.cpu().numpy(), ref)
    with pytest.raises(bfs.BfsError):
        g2.autotune(np.array([n], dtype=np.int32))
    g.close()
    g2.close()
    ctx.close()
