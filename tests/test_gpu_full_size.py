"""Parity at the benchmark sizes, in the launch configurations the benchmark
times: Kronecker scale 22 (edge factor 16, the headline graph and roots)
single-source -- default, direction-optimizing and CUDA-graph loops -- on
sampled roots, and the 64-root batched launches on the scale-24 Kronecker
and Erdos-Renyi graphs on sampled lanes, each compared element by element
with the oracle run on that root."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = bfs.Context(0)
    yield c
    c.close()


def test_scale22_single_source(ctx):
    off, col = graphgen.kronecker(22, 16, seed=22)
    roots = graphgen.pick_roots(off, 64, seed=3)
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    cases = [(int(roots[0]), 0, 0), (int(roots[37]), 0, 0), (int(roots[63]), 1, 0),
             (int(roots[5]), 0, bfs.BFS_GRAPH_LOOP), (int(roots[6]), 1, bfs.BFS_GRAPH_LOOP)]
    for r, direction, flags in cases:
        g.set_option(bfs.BFS_OPT_DIRECTION, direction)
        g.run(r, d, p, flags=flags)
        st = g.sync()
        ref, _, info = oracle.bfs(off, col, r)
        dist = d.cpu().numpy()
        assert np.array_equal(dist, ref), (r, direction, flags)
        assert oracle.check_tree(off, col, r, dist, p.cpu().numpy()) == []
        assert (st["levels"], st["reached"], st["edges_scanned"]) == \
            (info["levels"], info["reached"], info["edges_scanned"])
    g.close()


@pytest.mark.parametrize("name", ["kronecker", "erdos_renyi"])
def test_scale24_batched_sampled_lanes(ctx, name):
    if name == "kronecker":
        off, col = graphgen.kronecker(24, 16, seed=24)
    else:
        off, col = graphgen.erdos_renyi(24, 32, seed=25)
    roots = graphgen.pick_roots(off, 64, seed=3)
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    d = torch.empty((64, n), dtype=torch.int32, device="cuda")
    for direction in (0, 1):
        g.set_option(bfs.BFS_OPT_DIRECTION, direction)
        g.run_batch(roots, d)
        st = g.batch_sync()
        assert st["status"] == 0
        for lane in ((0, 63) if direction == 0 else (31,)):
            ref, _, _ = oracle.bfs(off, col, int(roots[lane]))
            assert np.array_equal(d[lane].cpu().numpy(), ref), (name, direction, lane)
    g.close()
