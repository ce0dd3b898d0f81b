"""ButterFly BFS (Algorithm 2) emulated with virtual compute nodes on one
GPU: distances bit-exact against the oracle for every node count and
fanout, every node's view identical, and the message accounting of
Section "Fanout & Trade-offs" (nodes * (r - 1) messages per round, receive
buffers within (r - 1) * V)."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402

CASES = [(1, 1), (2, 1), (4, 1), (16, 1), (4, 4), (16, 4), (8, 2), (27, 3)]


@pytest.fixture(scope="module")
def ctx():
    c = bfs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("nodes,fanout", CASES, ids=[f"P{p}_f{f}" for p, f in CASES])
def test_butterfly_matches_oracle(ctx, nodes, fanout):
    off, col = graphgen.kronecker(14, 8, seed=31)
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    radix = max(2, fanout)
    for r in graphgen.pick_roots(off, 3, seed=nodes * 7 + fanout):
        dist = torch.empty(n, dtype=torch.int32, device="cuda")
        st = g.run_butterfly(int(r), nodes, fanout, dist)
        ref, _, info = oracle.bfs(off, col, int(r))
        assert np.array_equal(dist.cpu().numpy(), ref)
        assert st["node_disagreements"] == 0
        assert st["levels"] == info["levels"]
        assert st["messages"] == st["levels"] * nodes * (radix - 1) * st["rounds_per_level"]
        assert st["max_round_buffer_entries"] <= (radix - 1) * n
    g.close()


@pytest.mark.parametrize("graph", ["path", "union", "caller_order"])
def test_butterfly_other_graphs(ctx, graph):
    flags = 0
    if graph == "path":
        off, col = G.path(500)
    elif graph == "union":
        off, col = G.disjoint_union(G.grid(30, 40), G.star(700))
    else:
        off, col = graphgen.kronecker(12, 8, seed=3)
        flags = bfs.BFS_UPLOAD_NO_RELABEL
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col, flags=flags)
    for r in (0, n // 2, n - 1):
        for nodes, fanout in ((8, 1), (16, 4)):
            dist = torch.empty(n, dtype=torch.int32, device="cuda")
            st = g.run_butterfly(r, nodes, fanout, dist)
            ref, _, _ = oracle.bfs(off, col, r)
            assert np.array_equal(dist.cpu().numpy(), ref)
            assert st["node_disagreements"] == 0
    g.close()


def test_butterfly_rejects_bad_node_counts(ctx):
    off, col = G.path(10)
    g = bfs.Graph(ctx, off, col)
    d = torch.empty(10, dtype=torch.int32, device="cuda")
    for nodes, fanout in ((6, 1), (8, 4), (0, 1)):
        with pytest.raises(bfs.BfsError):
            g.run_butterfly(0, nodes, fanout, d)
    g.close()


@pytest.mark.parametrize("graph", ["kron14", "path", "union", "er", "directed"])
def test_lrb_comparison_path_matches_oracle(ctx, graph):
    flags = 0
    if graph == "kron14":
        off, col = graphgen.kronecker(14, 16, seed=32)
    elif graph == "path":
        off, col = G.path(400)
    elif graph == "union":
        off, col = G.disjoint_union(G.grid(30, 40), G.star(3000))
    elif graph == "er":
        off, col = graphgen.erdos_renyi(13, 16, seed=33)
        flags = bfs.BFS_UPLOAD_NO_RELABEL
    else:
        off, col = G.random_graph(3000, 12000, 4, undirected=False)
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col, flags=flags)
    for r in (0, n // 2, n - 1):
        dist = torch.empty(n, dtype=torch.int32, device="cuda")
        st = g.run_lrb(r, dist)
        ref, _, info = oracle.bfs(off, col, r)
        assert np.array_equal(dist.cpu().numpy(), ref)
        assert st["levels"] == info["levels"] and st["kernels"] >= st["levels"] - 1
    g.close()
