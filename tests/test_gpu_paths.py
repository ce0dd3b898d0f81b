"""Shortest-path counts and weight-filtered traversal (bfs_run_paths) against
the oracle's Brandes forward phase: hops bit-exact; sigma bit-exact wherever
the oracle's count is below 2^53 (every term and partial sum of such a count
is then an integer below 2^53, so any addition order gives the same double),
elsewhere within the rounding bound levels x max in-degree x 2^-52; the
level, reached and scanned-entry counts equal.  Kronecker, Erdos-Renyi and
directed random graphs, weight filters (half the entries, one weight, an
empty range), a grid whose counts pass 2^53, a hub row spread over many
tiles, frontiers of degree-0 vertices, single-vertex and isolated-root
graphs, an arena context, the benchmark's scale-22 workload (8 roots, both
filters),
and the error paths (bad CSR, host memory)."""
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


def dev(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return torch.from_numpy(a).cuda() if a.size else torch.empty(0, dtype=torch.from_numpy(a).dtype,
                                                                 device="cuda")


def run(ctx, off, col, root, weight=None, lo=0, hi=0):
    n = len(off) - 1
    hops = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    sigma = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    w = None if weight is None else dev(weight, np.int32)
    st = ctx.run_paths(dev(off, np.int64), dev(col, np.int32), int(root), hops, sigma, w, lo, hi)
    return hops.cpu().numpy(), sigma.cpu().numpy(), st


def check(ctx, off, col, root, weight=None, lo=0, hi=0):
    hops, sigma, st = run(ctx, off, col, root, weight, lo, hi)
    eh, es, info = oracle.bfs_paths(off, col, int(root), weight, lo, hi)
    assert np.array_equal(hops, eh)
    exact = es < 2.0 ** 53
    assert np.array_equal(sigma[exact], es[exact])
    if not exact.all():
        indeg = np.bincount(np.asarray(col, dtype=np.int64), minlength=len(off) - 1).max()
        tol = info["levels"] * max(1, int(indeg)) * 2.0 ** -52
        assert np.allclose(sigma[~exact], es[~exact], rtol=tol, atol=0.0)
    assert st["levels"] == info["levels"]
    assert st["reached"] == info["reached"]
    assert st["edges_scanned"] == info["edges_scanned"]
    return st


def weights_for(col, seed, top=8):
    return np.random.default_rng(seed).integers(0, top, len(col)).astype(np.int32)


@pytest.mark.parametrize("scale,ef", [(14, 8), (16, 16)])
def test_paths_kronecker(ctx, scale, ef):
    off, col = graphgen.kronecker(scale, ef, seed=scale)
    for r in graphgen.pick_roots(off, 4, seed=ef):
        check(ctx, off, col, r)


def test_paths_other_graphs(ctx):
    off, col = graphgen.erdos_renyi(14, 16, seed=3)
    for r in graphgen.pick_roots(off, 3, seed=1):
        check(ctx, off, col, r)
    off, col = G.random_graph(3000, 9000, 5, undirected=False)
    for r in (0, 17, 2999):
        check(ctx, off, col, r)


@pytest.mark.parametrize("lo,hi", [(0, 3), (5, 5), (7, 0), (0, 7)])
def test_paths_weight_filter(ctx, lo, hi):
    off, col = graphgen.kronecker(14, 16, seed=9)
    w = weights_for(col, 11)
    for r in graphgen.pick_roots(off, 3, seed=lo * 8 + hi):
        st = check(ctx, off, col, r, w, lo, hi)
        if lo > hi:
            assert st["reached"] == 1 and st["levels"] == 1


def test_paths_grid_counts_beyond_2_53(ctx):
    rows, cols = 40, 50
    off, col = G.grid(rows, cols)
    check(ctx, off, col, 0)
    check(ctx, off, col, rows * cols // 2 + 7)
    # horizontal entries weigh 1, vertical ones 2: filter [1, 1] keeps row 0
    src = np.repeat(np.arange(rows * cols), np.diff(off))
    w = np.where(src // cols == col // cols, 1, 2).astype(np.int32)
    hops, sigma, st = run(ctx, off, col, 0, w, 1, 1)
    assert hops[:cols].tolist() == list(range(cols)) and np.all(hops[cols:] == -1)
    assert np.all(sigma[:cols] == 1.0) and np.all(sigma[cols:] == 0.0)
    off, col = G.hypercube(16)
    check(ctx, off, col, 0)


def test_paths_hub_rows_and_empty_frontiers(ctx):
    # a hub of 300,000 leaves: its row spans many 2048-entry tiles
    off, col = G.star(300_001)
    check(ctx, off, col, 0)
    check(ctx, off, col, 12345)
    # directed star: the level-1 frontier holds only degree-0 vertices
    off, col = G.from_edges(5000, np.zeros(4999, dtype=np.int64), np.arange(1, 5000),
                            undirected=False)
    check(ctx, off, col, 0)
    check(ctx, off, col, 4)
    # ragged: chains and stars of every size glued into one graph
    rng = np.random.default_rng(4)
    src, dst = [], []
    base = 0
    for size in rng.integers(1, 700, 60):
        hub = base
        leaves = np.arange(base + 1, base + 1 + size)
        src.append(np.full(size, hub))
        dst.append(leaves)
        src.append(leaves[:-1])
        dst.append(leaves[1:])
        base += size + 1
    src.append(np.arange(0, base - 1, 97))
    dst.append(np.arange(1, base, 97))
    off, col = G.from_edges(base, np.concatenate(src), np.concatenate(dst))
    for r in (0, base // 2, base - 1):
        check(ctx, off, col, r)


def test_paths_degenerate_graphs(ctx):
    off, col = np.array([0, 0], dtype=np.int64), np.zeros(0, dtype=np.int32)
    hops, sigma, st = run(ctx, off, col, 0)
    assert hops.tolist() == [0] and sigma.tolist() == [1.0]
    assert st == {"levels": 1, "reached": 1, "edges_scanned": 0}
    off, col = G.disjoint_union(G.path(4), G.from_edges(3, [], []))
    check(ctx, off, col, 5)
    check(ctx, off, col, 1)
    # a self-loop and a duplicated entry: 0 -> 0, 0 -> 1 twice, 1 -> 2
    off = np.array([0, 3, 4, 4], dtype=np.int64)
    col = np.array([0, 1, 1, 2], dtype=np.int32)
    hops, sigma, st = run(ctx, off, col, 0)
    assert hops.tolist() == [0, 1, 2] and sigma.tolist() == [1.0, 2.0, 2.0]
    check(ctx, off, col, 0)


def test_paths_arena_context():
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    with bfs.Context(0, arena=arena) as c:
        off, col = graphgen.kronecker(13, 8, seed=2)
        used0 = c.memory()[0]
        for r in graphgen.pick_roots(off, 2, seed=2):
            check(c, off, col, r)
        assert c.memory()[0] == used0  # scratch returned


def test_paths_bad_csr_is_an_error(ctx):
    off, col = G.path(6)
    bad = col.copy()
    bad[3] = 6                     # column index == n
    with pytest.raises(bfs.BfsError) as err:
        run(ctx, off, bad, 0)
    assert err.value.status == bfs.BFS_ERR_INVALID_GRAPH
    bad_off = off.copy()
    bad_off[-1] = len(col) + 5     # last row ends past nnz
    with pytest.raises(bfs.BfsError) as err:
        run(ctx, bad_off, col, 5)
    assert err.value.status == bfs.BFS_ERR_INVALID_GRAPH
    check(ctx, off, col, 0)        # the context is still usable


def test_paths_rejects_host_memory(ctx):
    off, col = G.path(8)
    n = len(off) - 1
    h_off = torch.from_numpy(off).pin_memory()
    d_col = dev(col, np.int32)
    hops = torch.empty(n, dtype=torch.int32, device="cuda")
    sigma = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = bfs._lib.lib().bfs_run_paths(ctx.handle, h_off.data_ptr(), d_col.data_ptr(), None, n,
                                      len(col), 0, 0, 0, hops.data_ptr(), sigma.data_ptr(), None,
                                      None)
    assert rc == bfs.BFS_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        ctx.run_paths(h_off, d_col, 0, hops, sigma)
    rc = bfs._lib.lib().bfs_run_paths(ctx.handle, dev(off, np.int64).data_ptr(), d_col.data_ptr(),
                                      None, n, len(col), 0, 0, n, hops.data_ptr(),
                                      sigma.data_ptr(), None, None)
    assert rc == bfs.BFS_ERR_ROOT_RANGE


def test_paths_scale22_bench_roots(ctx):
    """The benchmark's path-count workload: the headline graph, its first 8
    roots, every entry kept and weights 0-3 of uniform 0-7 kept."""
    from concurrent.futures import ThreadPoolExecutor

    from tests import fullsize as F
    off, col = F.graph(F.KRON_S22)
    roots = [int(r) for r in graphgen.pick_roots(off, 64, seed=F.ROOT_SEED)[:8]]
    w = weights_for(col, 5)
    cases = [(r, None, 0, 0) for r in roots] + [(r, w, 0, 3) for r in roots]
    with ThreadPoolExecutor(max_workers=8) as ex:
        refs = list(ex.map(lambda c: oracle.bfs_paths(off, col, c[0], c[1], c[2], c[3]), cases))
    d_off, d_col, d_w = dev(off, np.int64), dev(col, np.int32), dev(w, np.int32)
    n = len(off) - 1
    hops = torch.empty(n, dtype=torch.int32, device="cuda")
    sigma = torch.empty(n, dtype=torch.float64, device="cuda")
    for (r, wt, lo, hi), (eh, es, info) in zip(cases, refs):
        st = ctx.run_paths(d_off, d_col, r, hops, sigma, None if wt is None else d_w, lo, hi)
        assert np.array_equal(hops.cpu().numpy(), eh), (r, lo, hi)
        sg = sigma.cpu().numpy()
        exact = es < 2.0 ** 53
        assert np.array_equal(sg[exact], es[exact]), (r, lo, hi)
        if not exact.all():
            tol = info["levels"] * int(np.bincount(col, minlength=n).max()) * 2.0 ** -52
            assert np.allclose(sg[~exact], es[~exact], rtol=tol, atol=0.0)
        assert (st["levels"], st["reached"], st["edges_scanned"]) == \
            (info["levels"], info["reached"], info["edges_scanned"])
