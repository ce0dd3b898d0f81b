"""Failure detection without a GPU fault: the grid barrier's bounded wait.

The test hook makes the barrier expect one arrival more than the grid has,
so every CTA's wait runs out after the configured limit (a short one here),
the kernel records BFS_ERR_TIMEOUT and returns normally; the context stays
usable and the next traversal is correct."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


def test_barrier_wait_times_out_and_recovers():
    ctx = bfs.Context(0)
    off, col = graphgen.kronecker(12, 8, seed=3)
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    lib = bfs.load()
    assert lib.bfs_debug_set_barrier_test(g.handle, 1, 20_000_000) == 0  # 20 ms limit
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    g.run(0, d)
    with pytest.raises(bfs.BfsError) as e:
        g.sync()
    assert e.value.status == bfs.BFS_ERR_TIMEOUT
    # batched path too
    bd = torch.empty((4, n), dtype=torch.int32, device="cuda")
    g.run_batch(np.array([0, 1, 2, 3], dtype=np.int32), bd)
    with pytest.raises(bfs.BfsError) as e:
        g.batch_sync()
    assert e.value.status == bfs.BFS_ERR_TIMEOUT
    # back to normal
    assert lib.bfs_debug_set_barrier_test(g.handle, 0, 0) == 0
    root = int(graphgen.pick_roots(off, 1, seed=1)[0])
    g.run(root, d)
    st = g.sync()
    assert st["status"] == 0
    ref, _, _ = oracle.bfs(off, col, root)
    assert np.array_equal(d.cpu().numpy(), ref)
    torch.cuda.synchronize()
    g.close()
    ctx.close()
