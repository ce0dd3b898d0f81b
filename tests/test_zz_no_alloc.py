"""bfs_run_static: the traversal for callers that cannot allocate device
memory (a fixed memory plan owned by a framework or service, or code that
must not trigger the synchronisation cudaMalloc/cudaFree can imply).

Checks, through the C ABI, that two calls in a row give the distances of
the CPU oracle and of the regular entry point (bfs_graph_upload + bfs_run)
bit-exactly with valid parents, that graphs beyond the fixed scratch are
refused, and that a CSR failing the device-side check (a column index out
of range, decreasing offsets, a last offset beyond nnz) is reported as
BFS_ERR_INVALID_GRAPH with the outputs untouched.  Kept in a file that
pytest collects last; it passes alone in a fresh process as well as after
the other tests.
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
        d_oracle, _, info = oracle.bfs(off, col, r)
        d = dist.cpu().numpy()
        assert np.array_equal(d, d_oracle), f"call {call}: distances differ from the oracle"
        assert np.array_equal(d, d_ref), f"call {call}: distances differ from bfs_run"
        assert st["edges_scanned"] == info["edges_scanned"]
        assert st["levels"] == info["levels"]
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


def _bad_csr(kind):
    """A small valid CSR (path 0-1-2-...-9, both directions) made invalid in
    one way; buffers hold exactly n + 1 offsets and nnz columns."""
    n = 10
    rows = [[v - 1] * (v > 0) + [v + 1] * (v < n - 1) for v in range(n)]
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([u for r in rows for u in r], dtype=np.int32)
    if kind == "column_out_of_range":
        col[5] = n
    elif kind == "negative_column":
        col[3] = -1
    elif kind == "decreasing_offsets":
        off[4], off[5] = off[5], off[4]
    elif kind == "last_offset_beyond_nnz":
        col = col[:-2].copy()
    return off, col


@pytest.mark.parametrize("kind", ["column_out_of_range", "negative_column",
                                  "decreasing_offsets", "last_offset_beyond_nnz"])
def test_static_entry_rejects_invalid_csr(kind):
    off, col = _bad_csr(kind)
    n = len(off) - 1
    d_off = torch.from_numpy(off).cuda()
    d_col = torch.from_numpy(col).cuda()
    dist = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    parent = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_run_static(d_off, d_col, 0, dist, parent)
    assert e.value.status == bfs.BFS_ERR_INVALID_GRAPH
    assert b"CSR check failed" in bfs.load().bfs_last_error()
    assert torch.all(dist == 7).item() and torch.all(parent == 7).item()
    # the next call with a valid graph runs normally on the same scratch
    off2, col2 = _bad_csr("valid")
    d2 = torch.empty(n, dtype=torch.int32, device="cuda")
    st = bfs.bfs_run_static(torch.from_numpy(off2).cuda(), torch.from_numpy(col2).cuda(), 0, d2)
    assert st["status"] == 0
    assert np.array_equal(d2.cpu().numpy(), oracle.bfs(off2, col2, 0)[0])
