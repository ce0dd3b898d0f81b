"""Serving: queries on several resident graphs, submitted while others are
on the device, packed into batched launches.  Each result equals the
oracle (and hence the same query run alone), bit-exactly."""
from __future__ import annotations

import time

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    ctx = bfs.Context(0)
    graphs = []
    for scale, seed in ((12, 1), (13, 2), (14, 3)):
        off, col = graphgen.kronecker(scale, 16, seed=seed)
        graphs.append((off, col, bfs.Graph(ctx, off, col)))
    yield ctx, graphs
    for _, _, g in graphs:
        g.close()
    ctx.close()


def test_mixed_queries_match_alone(setup):
    ctx, graphs = setup
    srv = bfs.Server(ctx, 512 << 20, num_streams=3)
    gids = [srv.add_graph(g) for _, _, g in graphs]
    rng = np.random.default_rng(0)
    plan = []
    for i in range(150):
        gi = int(rng.integers(0, len(graphs)))
        off, col, _ = graphs[gi]
        root = int(graphgen.pick_roots(off, 1, seed=1000 + i)[0])
        plan.append((gi, root, np.full(len(off) - 1, -7, dtype=np.int32)))
    queries = []
    # first wave in a tight loop (queries pile up behind the busy slots and
    # get packed), second wave trickles in while the first is on the device
    for i, (gi, root, out) in enumerate(plan):
        queries.append((gi, root, out, srv.submit(gids[gi], root, out)))
        if i >= 100 and i % 10 == 0:
            time.sleep(0.001)
    for gi, root, out, t in queries:
        assert srv.wait(t, 30_000_000) == bfs.BFS_OK
        off, col, _ = graphs[gi]
        ref, _, _ = oracle.bfs(off, col, root)
        assert np.array_equal(out, ref)
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == 150 and st["failed"] == 0
    assert st["launches"] < 150, "queries on the same graph were never packed together"
    srv.close()


def test_budget_rejection_and_poll(setup):
    ctx, graphs = setup
    # one query on a 2^18-vertex graph needs > 4 MiB (two 8-byte lane
    # words per vertex alone), so a 1 MiB budget can never admit it
    off, col = graphgen.kronecker(18, 4, seed=9)
    big = bfs.Graph(ctx, off, col)
    srv = bfs.Server(ctx, 1 << 20, num_streams=1)
    gid = srv.add_graph(big)
    out = np.empty(len(off) - 1, dtype=np.int32)
    with pytest.raises(bfs.BfsError) as e:
        srv.submit(gid, 0, out)
    assert e.value.status == bfs.BFS_ERR_BUDGET
    srv.close()
    big.close()
    srv = bfs.Server(ctx, 256 << 20, num_streams=1)
    gid = srv.add_graph(graphs[0][2])
    off, col, _ = graphs[0]
    out = np.empty(len(off) - 1, dtype=np.int32)
    t = srv.submit(gid, 5, out)
    deadline = time.time() + 30
    while srv.poll(t) == bfs.BFS_PENDING and time.time() < deadline:
        time.sleep(0.0005)
    assert srv.poll(t) == bfs.BFS_OK
    ref, _, _ = oracle.bfs(off, col, 5)
    assert np.array_equal(out, ref)
    with pytest.raises(bfs.BfsError) as e:
        srv.poll(12345)
    assert e.value.status == bfs.BFS_ERR_NOT_FOUND
    srv.close()


def test_native_replay(setup):
    """bfs_server_replay submits a timed trace from native threads, reusing a
    few output buffers per graph; every query completes after its arrival and
    each buffer ends up holding its last query's row."""
    ctx, graphs = setup
    srv = bfs.Server(ctx, 512 << 20, num_streams=3)
    gids = [srv.add_graph(g) for _, _, g in graphs]
    rng = np.random.default_rng(7)
    nq = 120
    which = rng.integers(0, len(graphs), nq).astype(np.int32)
    roots = np.array([int(graphgen.pick_roots(graphs[w][0], 1, seed=2000 + i)[0])
                      for i, w in enumerate(which)], dtype=np.int32)
    arrival = time.monotonic_ns() + 5_000_000 + np.cumsum(rng.exponential(100_000, nq)).astype(np.int64)
    k = 3
    bufs = [np.full((k, len(off) - 1), -7, dtype=np.int32) for off, _, _ in graphs]
    done, status, slot = srv.replay(np.array(gids, dtype=np.int32)[which], roots, arrival, bufs,
                                    timeout_us=30_000_000)
    assert np.all(status == bfs.BFS_OK)
    assert np.all(done >= arrival)
    assert np.all((slot >= 0) & (slot < k))
    # each buffer holds the row of the last-completed query that used it
    for gi, (off, col, _) in enumerate(graphs):
        for sl in range(k):
            mine = np.nonzero((which == gi) & (slot == sl))[0]
            if len(mine) == 0:
                continue
            last = mine[np.argmax(done[mine])]
            ref, _, _ = oracle.bfs(off, col, int(roots[last]))
            assert np.array_equal(bufs[gi][sl], ref)
    assert srv.stats()["completed"] == nq
    srv.close()


def test_int8_and_int32_rows_in_one_stream(setup):
    """Queries asking for int8 rows (bfs_submit_rows with BFS_DIST_INT8) and
    for int32 rows, interleaved in one burst on three graphs: each row equals
    the oracle's distances, whichever launch and row type carried it."""
    ctx, graphs = setup
    srv = bfs.Server(ctx, 512 << 20, num_streams=3)
    gids = [srv.add_graph(g) for _, _, g in graphs]
    rng = np.random.default_rng(11)
    plan = []
    for i in range(120):
        gi = int(rng.integers(0, len(graphs)))
        off = graphs[gi][0]
        root = int(graphgen.pick_roots(off, 1, seed=3000 + i)[0])
        dt = torch.int8 if i % 2 else torch.int32
        out = torch.full((len(off) - 1,), -7, dtype=dt).pin_memory().numpy()
        plan.append((gi, root, out, srv.submit(gids[gi], root, out)))
    for gi, root, out, t in plan:
        assert srv.wait(t, 30_000_000) == bfs.BFS_OK
        off, col, _ = graphs[gi]
        assert np.array_equal(out.astype(np.int32), oracle.bfs(off, col, root)[0])
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == 120 and st["launches"] < 120
    srv.close()


def test_replays_with_int8_rows(setup):
    """The native replay and the one-at-a-time baseline with int8 rows."""
    ctx, graphs = setup
    srv = bfs.Server(ctx, 512 << 20, num_streams=3)
    gids = np.array([srv.add_graph(g) for _, _, g in graphs], dtype=np.int32)
    rng = np.random.default_rng(5)
    nq = 60
    which = rng.integers(0, len(graphs), nq).astype(np.int32)
    roots = np.array([int(graphgen.pick_roots(graphs[w][0], 1, seed=4000 + i)[0])
                      for i, w in enumerate(which)], dtype=np.int32)
    counts = np.bincount(which, minlength=len(graphs))
    arrival = time.monotonic_ns() + 5_000_000 + np.cumsum(rng.exponential(50_000, nq)).astype(np.int64)
    bufs = [np.full((int(c) + 1, len(off) - 1), -7, dtype=np.int8) for c, (off, _, _) in
            zip(counts, graphs)]
    done, status, slot = srv.replay(gids[which], roots, arrival, bufs, timeout_us=30_000_000)
    assert np.all(status == bfs.BFS_OK)
    srv.close()
    arrival = time.monotonic_ns() + 5_000_000 + np.cumsum(rng.exponential(50_000, nq)).astype(np.int64)
    one = [np.full((1, len(off) - 1), -7, dtype=np.int8) for off, _, _ in graphs]
    done1, status1 = bfs.bfs_replay_single([g.handle for _, _, g in graphs], which, roots,
                                           arrival, one)
    assert np.all(status1 == bfs.BFS_OK) and np.all(done1 >= arrival)
    # the last query of each graph is the one left in its single row
    for gi, (off, col, _) in enumerate(graphs):
        mine = np.nonzero(which == gi)[0]
        if len(mine):
            last = mine[-1]
            assert np.array_equal(one[gi][0].astype(np.int32), oracle.bfs(off, col, int(roots[last]))[0])
