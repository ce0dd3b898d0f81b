"""The level loop captured as a CUDA graph (BFS_GRAPH_LOOP): a conditional
while node repeats the level kernels on the device.  Results must equal the
oracle (and the persistent launch) for single-source and batched runs; the
instantiated graph is reused across roots and rebuilt when buffers or
settings change."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = bfs.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def kron15():
    off, col = graphgen.kronecker(15, 16, seed=31)
    return off, col, graphgen.pick_roots(off, 12, seed=32)


def check_plain(off, col, root, dist, parent, st):
    ref, _, info = oracle.bfs(off, col, root)
    assert np.array_equal(dist, ref)
    assert oracle.check_tree(off, col, root, dist, parent) == []
    assert st["status"] == 0
    assert (st["levels"], st["reached"], st["edges_scanned"]) == \
        (info["levels"], info["reached"], info["edges_scanned"])


def test_plain_graph_loop_reuse_and_rebuild(ctx, kron15):
    off, col, roots = kron15
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:  # same buffers: one graph, new roots each time
        g.run(int(r), d, p, flags=bfs.BFS_GRAPH_LOOP)
        check_plain(off, col, int(r), d.cpu().numpy(), p.cpu().numpy(), g.sync())
    d2 = torch.empty(n, dtype=torch.int32, device="cuda")  # new buffers: rebuilt
    g.run(int(roots[0]), d2, None, flags=bfs.BFS_GRAPH_LOOP)
    ref, _, _ = oracle.bfs(off, col, int(roots[0]))
    assert np.array_equal(d2.cpu().numpy(), ref)
    g.set_option(bfs.BFS_OPT_DIRECTION, 1)  # settings change: rebuilt
    for r in roots[:4]:
        g.run(int(r), d, p, flags=bfs.BFS_GRAPH_LOOP)
        st = g.sync()
        check_plain(off, col, int(r), d.cpu().numpy(), p.cpu().numpy(), st)
        assert st["bottom_up_levels"] > 0
    h = np.empty(n, dtype=np.int32)
    hp = np.empty(n, dtype=np.int32)
    g.run(int(roots[1]), h, hp, flags=bfs.BFS_GRAPH_LOOP)
    check_plain(off, col, int(roots[1]), h, hp, g.sync())
    with pytest.raises(bfs.BfsError):
        g.run(int(roots[0]), d, p, flags=bfs.BFS_GRAPH_LOOP | bfs.BFS_HOST_LOOP)
    g.close()


@pytest.mark.parametrize("name,graph,roots", [
    ("path", G.path(600), [0, 300]),
    ("star", G.star(2000), [0, 5]),
    ("union", G.disjoint_union(G.path(50), G.star(300)), [3, 60]),
    ("single", (np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32)), [0]),
])
def test_plain_graph_loop_small_graphs(ctx, name, graph, roots):
    off, col = graph
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:
        g.run(int(r), d, p, flags=bfs.BFS_GRAPH_LOOP)
        check_plain(off, col, int(r), d.cpu().numpy(), p.cpu().numpy(), g.sync())
    g.close()


@pytest.mark.parametrize("k,int8", [(1, False), (16, False), (64, False), (64, True)])
def test_batched_graph_loop(ctx, kron15, k, int8):
    off, col, _ = kron15
    n = len(off) - 1
    roots = graphgen.pick_roots(off, k, seed=40 + k)
    g = bfs.Graph(ctx, off, col)
    dt = torch.int8 if int8 else torch.int32
    flags = bfs.BFS_GRAPH_LOOP | (bfs.BFS_DIST_INT8 if int8 else 0)
    ref, _ = oracle.bfs_multi(off, col, roots)
    for _ in range(2):  # the second run reuses the instantiated graph
        d = torch.empty((k, n), dtype=dt, device="cuda")
        g.run_batch(roots, d, flags=flags)
        st = g.batch_sync()
        assert st["status"] == 0
        assert np.array_equal(d.cpu().numpy().astype(np.int32), ref)
    pd = torch.empty((k, n), dtype=dt, device="cuda")
    g.run_batch(roots, pd, flags=(bfs.BFS_DIST_INT8 if int8 else 0))
    pst = g.batch_sync()
    assert (pst["levels"], pst["reached"], pst["edges_scanned"]) == \
        (st["levels"], st["reached"], st["edges_scanned"])
    g.close()


def test_batched_graph_loop_depth_limit(ctx):
    off, col = G.path(300)
    g = bfs.Graph(ctx, off, col)
    d = torch.empty((2, 300), dtype=torch.int8, device="cuda")
    with pytest.raises(bfs.BfsError) as ei:
        g.run_batch(np.array([0, 1], dtype=np.int32), d, flags=bfs.BFS_GRAPH_LOOP | bfs.BFS_DIST_INT8)
        g.batch_sync()
    assert ei.value.status == bfs.BFS_ERR_DEPTH_OVERFLOW
    d32 = torch.empty((2, 300), dtype=torch.int32, device="cuda")
    g.run_batch(np.array([0, 299], dtype=np.int32), d32, flags=bfs.BFS_GRAPH_LOOP)
    g.batch_sync()
    ref, _ = oracle.bfs_multi(off, col, np.array([0, 299], dtype=np.int32))
    assert np.array_equal(d32.cpu().numpy(), ref)
    g.close()
