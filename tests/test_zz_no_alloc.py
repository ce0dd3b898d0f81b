"""bfs_run_static: the traversal for callers that cannot allocate device
memory (a fixed memory plan owned by a framework or service, or code that
must not trigger the synchronisation cudaMalloc/cudaFree can imply).

Checks, through the C ABI, that two calls in a row give the same distances
as the regular entry point (bfs_graph_upload + bfs_run) bit-exactly and
valid parents, and that graphs beyond the fixed scratch are refused.  Kept
in a file that pytest collects last; it passes alone in a fresh process as
well as after the other tests.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


def _regular(off, col, root):
    ctx = bfs.Context(0)
    g = bfs.Graph(ctx, off, col)
    n = len(off) - 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    g.run(int(root), d, p)
    st = g.sync()
    out = d.cpu().numpy(), p.cpu().numpy(), st
    g.close()
    ctx.close()
    return out


@pytest.mark.parametrize("graph", ["kron16", "er14"])
def test_static_entry_matches_regular_entry_two_calls(graph):
    if graph == "kron16":
        off, col = graphgen.kronecker(16, 8, seed=1)
    else:
        off, col = graphgen.erdos_renyi(14, 16, seed=2)
    n = len(off) - 1
    d_off = torch.from_numpy(off).cuda()
    d_col = torch.from_numpy(col).cuda()
    roots = graphgen.pick_roots(off, 2, seed=12)
    for call in range(2):  # two calls in a row share the fixed scratch
        r = int(roots[call])
        dist = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        parent = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        st = bfs.bfs_run_static(d_off, d_col, r, dist, parent)
        d_ref, _, st_ref = _regular(off, col, r)
        d = dist.cpu().numpy()
        assert np.array_equal(d, d_ref), f"call {call}: distances differ from bfs_run"
        assert oracle.check_tree(off, col, r, d, parent.cpu().numpy()) == []
        assert st["status"] == 0
        assert (st["levels"], st["reached"], st["edges_scanned"]) == \
            (st_ref["levels"], st_ref["reached"], st_ref["edges_scanned"])


def test_static_entry_rejects_oversized_graphs():
    n = (1 << 19) + 1
    d_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    d_col = torch.zeros(16, dtype=torch.int32, device="cuda")
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_run_static(d_off, d_col[:0], 0, dist)
    assert e.value.status == bfs.BFS_ERR_UNSUPPORTED
    assert b"fixed scratch" in bfs.load().bfs_last_error()
