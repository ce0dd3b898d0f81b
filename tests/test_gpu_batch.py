"""GPU parity of the 64-lane batched traversal: row i of the batched
distances equals the oracle's BFS from roots[i], bit-exactly, for int32 and
int8 distances, device and host outputs, duplicate roots, and both the
device-side and host-driven level loops."""
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
def kron14():
    off, col = graphgen.kronecker(14, 8, seed=11)
    return off, col


def batch_gpu(g, n, roots, dtype=torch.int32, flags=0):
    d = torch.empty((len(roots), n), dtype=dtype, device="cuda")
    g.run_batch(roots, d, flags=flags)
    st = g.batch_sync()
    return d.cpu().numpy(), st


def expected(off, col, roots):
    ref, scanned = oracle.bfs_multi(off, col, roots)
    return ref, scanned


@pytest.mark.parametrize("k", [1, 7, 32, 33, 64])
def test_batch_rows_equal_oracle(ctx, kron14, k):
    off, col = kron14
    roots = graphgen.pick_roots(off, k, seed=100 + k)
    g = bfs.Graph(ctx, off, col)
    d, st = batch_gpu(g, len(off) - 1, roots)
    ref, scanned = expected(off, col, roots)
    assert np.array_equal(d, ref)
    assert st["status"] == 0
    assert st["edges_scanned"] == int(scanned.sum())
    assert st["reached"] == int(np.count_nonzero(ref >= 0))
    g.close()


def test_batch_duplicate_roots_and_unreachable(ctx):
    off, col = G.disjoint_union(G.grid(30, 30), G.star(500))
    roots = np.array([0, 0, 950, 899, 0, 950, 450, 901] * 8, dtype=np.int32)
    g = bfs.Graph(ctx, off, col)
    d, st = batch_gpu(g, len(off) - 1, roots)
    ref, _ = expected(off, col, roots)
    assert np.array_equal(d, ref)
    assert np.array_equal(d[0], d[1]) and np.array_equal(d[0], d[4])
    g.close()


@pytest.mark.parametrize("bins", [None, (1, 2, 1024, 1024), (1 << 20, (1 << 20) + 1, 1024, 8192),
                                  (4, 64, 128, 1024)])
def test_batch_bins(ctx, kron14, bins):
    off, col = kron14
    roots = graphgen.pick_roots(off, 64, seed=5)
    g = bfs.Graph(ctx, off, col)
    if bins:
        g.set_bins(*bins)
    d, _ = batch_gpu(g, len(off) - 1, roots)
    ref, _ = expected(off, col, roots)
    assert np.array_equal(d, ref)
    g.close()


def test_batch_int8_host_loop_and_host_output(ctx, kron14):
    off, col = kron14
    n = len(off) - 1
    roots = graphgen.pick_roots(off, 40, seed=6)
    ref, _ = expected(off, col, roots)
    g = bfs.Graph(ctx, off, col)
    d8, _ = batch_gpu(g, n, roots, dtype=torch.int8)
    assert np.array_equal(d8.astype(np.int32), ref)
    dl, st = batch_gpu(g, n, roots, flags=bfs.BFS_HOST_LOOP)
    assert np.array_equal(dl, ref)
    assert st["levels"] == int(ref.max()) + 1
    h = np.empty((len(roots), n), dtype=np.int32)
    g.run_batch(roots, h)
    assert np.array_equal(h, ref)
    g.close()


def test_batch_int8_depth_overflow(ctx):
    off, col = G.path(200)
    g = bfs.Graph(ctx, off, col)
    d = torch.empty((1, 200), dtype=torch.int8, device="cuda")
    g.run_batch(np.array([0], dtype=np.int32), d)
    with pytest.raises(bfs.BfsError) as e:
        g.batch_sync()
    assert e.value.status == bfs.BFS_ERR_DEPTH_OVERFLOW
    # shallow enough from the middle: levels <= 100
    g.run_batch(np.array([100], dtype=np.int32), d)
    g.batch_sync()
    ref, _ = expected(off, col, [100])
    assert np.array_equal(d.cpu().numpy().astype(np.int32), ref)
    g.close()


def test_batch_deep_graph_int32(ctx):
    # levels beyond 254 take the direct-write path of the level records
    off, col = G.path(700)
    roots = np.array([0, 350, 699, 0], dtype=np.int32)
    g = bfs.Graph(ctx, off, col)
    d, st = batch_gpu(g, 700, roots)
    ref, _ = expected(off, col, roots)
    assert np.array_equal(d, ref)
    assert st["levels"] == 700
    dl, _ = batch_gpu(g, 700, roots, flags=bfs.BFS_HOST_LOOP)
    assert np.array_equal(dl, ref)
    g.close()


@pytest.mark.parametrize("dtype", [torch.int32, torch.int8])
def test_batch_row_layouts(ctx, dtype):
    # the result rows are written four vertices per store when every row
    # start is aligned (n a multiple of 4, rows 16-byte aligned) and one
    # value per store otherwise: n = 702 and rows starting one element
    # past an aligned address take the second form
    for off, col in (G.grid(27, 26), graphgen.kronecker(10, 8, seed=5)):
        n = len(off) - 1
        roots = graphgen.pick_roots(off, 9, seed=7)
        ref, _ = expected(off, col, roots)
        g = bfs.Graph(ctx, off, col)
        flat = torch.empty(len(roots) * n + 1, dtype=dtype, device="cuda")
        rows = flat[1:].view(len(roots), n)
        g.run_batch(roots, rows)
        g.batch_sync()
        assert np.array_equal(rows.cpu().numpy().astype(np.int32), ref)
        aligned, _ = batch_gpu(g, n, roots, dtype=dtype)
        assert np.array_equal(aligned.astype(np.int32), ref)
        g.close()


def test_batch_equals_plain_runs(ctx):
    off, col = graphgen.erdos_renyi(13, 16, seed=8)
    n = len(off) - 1
    roots = graphgen.pick_roots(off, 64, seed=9)
    g = bfs.Graph(ctx, off, col)
    d, _ = batch_gpu(g, n, roots)
    for i in range(0, 64, 9):
        one = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(int(roots[i]), one)
        g.sync()
        assert np.array_equal(d[i], one.cpu().numpy())
    g.close()


def test_batch_bad_arguments(ctx):
    off, col = G.path(10)
    g = bfs.Graph(ctx, off, col)
    d = torch.empty((65, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        g.run_batch(np.zeros(65, dtype=np.int32), d)
    assert e.value.status == bfs.BFS_ERR_INVALID_ARG
    with pytest.raises(bfs.BfsError) as e:
        g.run_batch(np.array([3, 10], dtype=np.int32), d[:2])
    assert e.value.status == bfs.BFS_ERR_ROOT_RANGE
    g.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("k", [1, 17, 64])
def test_batch_direction_optimizing(ctx, kron14, mode, k):
    """Batched bottom-up levels (frontier lane sets of the neighbours ORed
    until every missing lane is found) give the oracle's rows."""
    off, col = kron14
    roots = graphgen.pick_roots(off, k, seed=300 + k)
    g = bfs.Graph(ctx, off, col)
    g.set_option(bfs.BFS_OPT_DIRECTION, mode)
    ref, _ = expected(off, col, roots)
    for flags in (0, bfs.BFS_GRAPH_LOOP):
        d, st = batch_gpu(g, len(off) - 1, roots, flags=flags)
        assert np.array_equal(d, ref)
        if mode == 2:
            assert st["bottom_up_levels"] > 0
    d8, _ = batch_gpu(g, len(off) - 1, roots, dtype=torch.int8, flags=bfs.BFS_DIST_INT8)
    assert np.array_equal(d8.astype(np.int32), ref)
    g.set_option(bfs.BFS_OPT_DIRECTION, 0)
    d0, st0 = batch_gpu(g, len(off) - 1, roots)
    assert np.array_equal(d0, ref) and st0["bottom_up_levels"] == 0
    g.close()


def test_batch_bottom_up_other_graphs(ctx):
    for name, (off, col) in (("grid", G.grid(30, 40)), ("union", G.disjoint_union(G.path(40), G.star(200))),
                             ("er", G.random_graph(3000, 12000, seed=9))):
        n = len(off) - 1
        roots = np.array([0, 1, n // 2, n - 1, 0], dtype=np.int32)
        g = bfs.Graph(ctx, off, col)
        g.set_option(bfs.BFS_OPT_DIRECTION, 2)
        d, _ = batch_gpu(g, n, roots)
        ref, _ = expected(off, col, roots)
        assert np.array_equal(d, ref), name
        g.close()
