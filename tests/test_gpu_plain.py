"""GPU parity of the single-source traversal against the CPU oracle.

Distances must match bit-exactly; parents are accepted when they satisfy
the Graph500-style invariants (several parents are valid).  Every case
goes through the C ABI.  Bin thresholds and chunk sizes are varied so
that each expansion path (warp gather, warp per vertex, CTA chunks, heavy
vertices split over many CTAs) carries whole traversals on its own.
"""
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


def run_gpu(g, n, root, flags=0, host=False):
    if host:
        dist = np.empty(n, dtype=np.int32)
        parent = np.empty(n, dtype=np.int32)
        g.run(root, dist, parent, flags=flags)
        return dist, parent, g.sync()
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    g.run(root, dist, parent, flags=flags)
    st = g.sync()
    return dist.cpu().numpy(), parent.cpu().numpy(), st


def assert_parity(off, col, root, dist, parent, stats, undirected=True):
    d_ref, _, info = oracle.bfs(off, col, root)
    assert np.array_equal(dist, d_ref), f"root {root}: {np.count_nonzero(dist != d_ref)} distances differ"
    assert oracle.check_tree(off, col, root, dist, parent, undirected=undirected) == []
    assert stats["status"] == 0
    assert stats["reached"] == info["reached"]
    assert stats["edges_scanned"] == info["edges_scanned"]
    assert stats["levels"] == info["levels"]


SMALL = [
    ("path", G.path(300), [0, 150, 299]),
    ("cycle", G.cycle(257), [0, 100]),
    ("star", G.star(5000), [0, 17]),
    ("grid", G.grid(40, 70), [0, 1234]),
    ("tree", G.binary_tree(4095), [0, 2047]),
    ("union", G.disjoint_union(G.path(50), G.star(300)), [3, 60]),
    ("complete", G.complete(200), [5]),
    ("isolated_root", G.disjoint_union((np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32)),
                                       G.cycle(10)), [0]),
]


@pytest.mark.parametrize("name,graph,roots", SMALL, ids=[s[0] for s in SMALL])
def test_closed_form_graphs(ctx, name, graph, roots):
    off, col = graph
    g = bfs.Graph(ctx, off, col)
    for r in roots:
        dist, parent, st = run_gpu(g, len(off) - 1, r)
        assert_parity(off, col, r, dist, parent, st)
    g.close()


def test_single_vertex_graph(ctx):
    off = np.zeros(2, dtype=np.int64)
    col = np.zeros(0, dtype=np.int32)
    g = bfs.Graph(ctx, off, col)
    dist, parent, st = run_gpu(g, 1, 0)
    assert dist.tolist() == [0] and parent.tolist() == [0]
    assert st["levels"] == 1 and st["reached"] == 1 and st["edges_scanned"] == 0
    g.close()


def test_directed_graph(ctx):
    off, col = G.random_graph(3000, 9000, 5, undirected=False)
    g = bfs.Graph(ctx, off, col)
    for r in (0, 7, 2999):
        dist, parent, st = run_gpu(g, 3000, r)
        assert_parity(off, col, r, dist, parent, st, undirected=False)
    g.close()


@pytest.fixture(scope="module")
def kron16():
    off, col = graphgen.kronecker(16, 8, seed=1)
    return off, col, graphgen.pick_roots(off, 16, seed=2)


BIN_SETTINGS = [
    ("default", None),
    ("all_small", (1 << 20, (1 << 20) + 1, 1024, 8192)),
    ("all_warp", (1, 1 << 20, 128, 8192)),
    ("all_cta", (1, 2, 1024, 1024)),
    ("tiny_chunks", (8, 64, 128, 1024)),
    ("wide_chunks", (64, 8192, 4096, 32768)),
]


@pytest.mark.parametrize("name,bins", BIN_SETTINGS, ids=[b[0] for b in BIN_SETTINGS])
def test_kron16_all_roots_bins(ctx, kron16, name, bins):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    if bins:
        g.set_bins(*bins)
    for r in roots:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
    g.close()


def test_relabelled_and_caller_order_uploads_agree(ctx, kron16):
    off, col, roots = kron16
    g1 = bfs.Graph(ctx, off, col)
    g2 = bfs.Graph(ctx, off, col, flags=bfs.BFS_UPLOAD_NO_RELABEL)
    assert g1.info()["relabelled"] == 1 and g2.info()["relabelled"] == 0
    assert g1.info()["max_degree"] == g2.info()["max_degree"] == int(np.diff(off).max())
    for r in roots[:8]:
        d1, p1, s1 = run_gpu(g1, len(off) - 1, int(r))
        d2, p2, s2 = run_gpu(g2, len(off) - 1, int(r))
        assert_parity(off, col, int(r), d1, p1, s1)
        assert_parity(off, col, int(r), d2, p2, s2)
    g1.close()
    g2.close()


@pytest.mark.parametrize("name,bins", BIN_SETTINGS[1:4], ids=[b[0] for b in BIN_SETTINGS[1:4]])
def test_caller_order_bins(ctx, kron16, name, bins):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col, flags=bfs.BFS_UPLOAD_NO_RELABEL)
    g.set_bins(*bins)
    for r in roots[:6]:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
    g.close()


@pytest.mark.parametrize("hot_words", [0, 4, 1024, 16384])
def test_shared_memory_hot_bitmap(ctx, kron16, hot_words):
    # min edges 0: every level takes the shared-memory copy path
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    g.set_option(bfs.BFS_OPT_HOT_WORDS, hot_words)
    g.set_option(bfs.BFS_OPT_HOT_MIN_EDGES, 0)
    for r in roots[:8]:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
        d2, p2, s2 = run_gpu(g, len(off) - 1, int(r), flags=bfs.BFS_HOST_LOOP)
        assert_parity(off, col, int(r), d2, p2, s2)
    g.close()


@pytest.mark.parametrize("div", [1 << 20, 16, 2])
def test_bitmap_frontier_top_down(ctx, kron16, div):
    # 2^20: every level with more than n / 2^20 frontier vertices (all of
    # them here) walks the frontier bitmap
    off, col, roots = kron16
    for upflags in (0, bfs.BFS_UPLOAD_NO_RELABEL):
        g = bfs.Graph(ctx, off, col, flags=upflags)
        g.set_option(bfs.BFS_OPT_BITMAP_FRONTIER, div)
        for r in roots[:8]:
            dist, parent, st = run_gpu(g, len(off) - 1, int(r))
            assert_parity(off, col, int(r), dist, parent, st)
            d2, p2, s2 = run_gpu(g, len(off) - 1, int(r), flags=bfs.BFS_HOST_LOOP)
            assert_parity(off, col, int(r), d2, p2, s2)
        g.set_option(bfs.BFS_OPT_DIRECTION, 1)
        for r in roots[8:12]:
            dist, parent, st = run_gpu(g, len(off) - 1, int(r))
            assert_parity(off, col, int(r), dist, parent, st)
        g.close()


def test_bitmap_frontier_small_graphs(ctx):
    for off, col in (G.grid(50, 70), G.disjoint_union(G.path(300), G.star(3000)),
                     G.random_graph(5000, 20000, 3, undirected=False)):
        g = bfs.Graph(ctx, off, col)
        g.set_option(bfs.BFS_OPT_BITMAP_FRONTIER, 1 << 20)
        n = len(off) - 1
        und = np.array_equal(np.sort(col), np.sort(col))  # always true; directed flag below
        for r in (0, n // 3, n - 1):
            dist, parent, st = run_gpu(g, n, r)
            d_ref, _, _ = oracle.bfs(off, col, r)
            assert np.array_equal(dist, d_ref)
        g.close()


DIRECTIONS = [
    ("do_default", 1, None, None, 0),
    ("do_eager", 1, 1 << 20, 1, 0),      # switches to bottom-up as early as possible
    ("do_caller_order", 1, None, None, bfs.BFS_UPLOAD_NO_RELABEL),
    ("bottom_up_always", 2, None, None, 0),
    ("bottom_up_always_caller_order", 2, None, None, bfs.BFS_UPLOAD_NO_RELABEL),
]


@pytest.mark.parametrize("name,mode,alpha,beta,upflags", DIRECTIONS, ids=[d[0] for d in DIRECTIONS])
def test_direction_optimizing(ctx, kron16, name, mode, alpha, beta, upflags):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col, flags=upflags)
    g.set_option(bfs.BFS_OPT_DIRECTION, mode)
    if alpha:
        g.set_option(bfs.BFS_OPT_DO_ALPHA, alpha)
    if beta:
        g.set_option(bfs.BFS_OPT_DO_BETA, beta)
    bu_seen = 0
    for r in roots[:10]:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
        bu_seen += st["bottom_up_levels"]
        d2, p2, s2 = run_gpu(g, len(off) - 1, int(r), flags=bfs.BFS_HOST_LOOP)
        assert_parity(off, col, int(r), d2, p2, s2)
        assert s2["bottom_up_levels"] == st["bottom_up_levels"]
    if mode == 2:
        assert bu_seen > 0
    g.close()


@pytest.mark.parametrize("graph", ["grid", "union", "directed", "er"])
def test_bottom_up_always_other_graphs(ctx, graph):
    if graph == "grid":
        off, col = G.grid(60, 80)
    elif graph == "union":
        off, col = G.disjoint_union(G.path(100), G.star(2000))
    elif graph == "directed":
        off, col = G.random_graph(4000, 16000, 9, undirected=False)
    else:
        off, col = graphgen.erdos_renyi(14, 16, seed=5)
    g = bfs.Graph(ctx, off, col)
    n = len(off) - 1
    if graph == "directed":
        # bottom-up needs every edge stored both ways; the upload's symmetry
        # test rejects the option on a directed graph
        with pytest.raises(bfs.BfsError) as e:
            g.set_option(bfs.BFS_OPT_DIRECTION, 2)
        assert e.value.status == bfs.BFS_ERR_UNSUPPORTED
        g.close()
        return
    g.set_option(bfs.BFS_OPT_DIRECTION, 2)
    for r in (0, n // 2, n - 1):
        dist, parent, st = run_gpu(g, n, r)
        assert_parity(off, col, r, dist, parent, st)
    g.close()


def test_kron16_host_loop_and_host_outputs(ctx, kron16):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    for r in roots[:6]:
        d1, p1, s1 = run_gpu(g, len(off) - 1, int(r), flags=bfs.BFS_HOST_LOOP)
        assert_parity(off, col, int(r), d1, p1, s1)
        d2, p2, s2 = run_gpu(g, len(off) - 1, int(r), host=True)
        assert_parity(off, col, int(r), d2, p2, s2)
    g.close()


def test_match_any_visited_update(ctx, kron16):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    g.set_option(bfs.BFS_OPT_WARP_AGGREGATE, 1)
    for r in roots:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
    g.close()


def test_er_graph(ctx):
    off, col = graphgen.erdos_renyi(15, 32, seed=3)
    g = bfs.Graph(ctx, off, col)
    for r in graphgen.pick_roots(off, 6, seed=4):
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
    g.close()


def test_device_pointer_upload_and_arena(kron16):
    off, col, roots = kron16
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    c = bfs.Context(0, arena=arena)
    g = bfs.Graph(c, torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
    used, cap = c.memory()
    assert 0 < used <= cap == 256 << 20
    for r in roots[:3]:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
    g.close()
    assert c.memory()[0] == 0
    c.close()


def test_errors(ctx):
    off, col = G.path(10)
    g = bfs.Graph(ctx, off, col)
    d = np.empty(10, dtype=np.int32)
    with pytest.raises(bfs.BfsError) as e:
        g.run(10, d)
    assert e.value.status == bfs.BFS_ERR_ROOT_RANGE
    with pytest.raises(bfs.BfsError) as e:
        g.run(-1, d)
    assert e.value.status == bfs.BFS_ERR_ROOT_RANGE
    g.close()
    bad = col.copy()
    bad[3] = 10
    with pytest.raises(bfs.BfsError) as e:
        bfs.Graph(ctx, off, bad)
    assert e.value.status == bfs.BFS_ERR_INVALID_GRAPH
    off2 = off.copy()
    off2[5], off2[6] = off2[6], off2[5]
    with pytest.raises(bfs.BfsError) as e:
        bfs.Graph(ctx, off2, col)
    assert e.value.status == bfs.BFS_ERR_INVALID_GRAPH
    off3 = off.copy()
    off3[-1] += 1
    with pytest.raises(bfs.BfsError) as e:
        bfs.Graph(ctx, off3, col)
    assert e.value.status == bfs.BFS_ERR_INVALID_GRAPH


def test_stream_ordering_on_torch_stream(ctx, kron16):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    s = torch.cuda.Stream()
    n = len(off) - 1
    outs = []
    with torch.cuda.stream(s):
        for r in roots[:4]:
            d = torch.empty(n, dtype=torch.int32, device="cuda")
            g.run(int(r), d, None, stream=s)
            outs.append(d.clone())
    s.synchronize()
    for r, d in zip(roots[:4], outs):
        d_ref, _, _ = oracle.bfs(off, col, int(r))
        assert np.array_equal(d.cpu().numpy(), d_ref)
    g.close()


def test_chunk_sizes_must_be_powers_of_two(ctx, kron16):
    off, col, _ = kron16
    g = bfs.Graph(ctx, off, col)
    for bins in ((32, 4096, 384, 2048), (32, 4096, 512, 3072), (32, 4096, 64, 2048)):
        with pytest.raises(bfs.BfsError):
            g.set_bins(*bins)
    g.set_bins(32, 4096, 256, 1024)
    g.close()


def test_l2_prefetch_option(ctx, kron16):
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    g.set_option(bfs.BFS_OPT_L2_PREFETCH, 1)
    for bins in (None, (1, 2, 1024, 1024), (1, 1 << 20, 128, 8192)):
        if bins:
            g.set_bins(*bins)
        for r in roots[:4]:
            dist, parent, st = run_gpu(g, len(off) - 1, int(r))
            assert_parity(off, col, int(r), dist, parent, st)
    with pytest.raises(bfs.BfsError):
        g.set_option(bfs.BFS_OPT_L2_PREFETCH, 2)
    g.close()


def test_level_timeline(ctx, kron16):
    """The timeline stamps init, seed and every level in order; levels match."""
    off, col, roots = kron16
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    stamps = torch.zeros(64, dtype=torch.int64, device="cuda")
    bfs.bfs_debug_set_timeline(g.handle, stamps)
    dist, parent, st = run_gpu(g, n, int(roots[0]))
    assert_parity(off, col, int(roots[0]), dist, parent, st)
    t = stamps.cpu().numpy()
    k = 3 + st["levels"]
    assert np.all(t[:k] > 0) and np.all(np.diff(t[:k]) >= 0)
    assert np.all(t[k:] == 0)
    # batched: [3 + 2L] after the expansion, [4 + 2L] after the sweep of level L
    stamps.zero_()
    rts = np.asarray(roots[:8], dtype=np.int32)
    d = torch.empty((len(rts), n), dtype=torch.int32, device="cuda")
    g.run_batch(rts, d)
    bst = g.batch_sync()
    t = stamps.cpu().numpy()
    kb = 3 + 2 * (bst["levels"] - 1)
    assert np.all(t[:kb] > 0) and np.all(np.diff(t[:kb]) >= 0)
    bfs.bfs_debug_set_timeline(g.handle, None)
    stamps.zero_()
    run_gpu(g, n, int(roots[1]))
    assert np.all(stamps.cpu().numpy() == 0)
    with pytest.raises(bfs.BfsError):
        bfs.bfs_debug_set_timeline(g.handle, torch.zeros(2, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        bfs.bfs_debug_set_timeline(g.handle, torch.zeros(8, dtype=torch.int64))
    g.close()


@pytest.mark.parametrize("bins", [None, (1, 2, 1024, 1024), (4, 64, 128, 2048)])
def test_tma_staged_heavy_runs(ctx, kron16, bins):
    """Bin-2 column runs staged in shared memory by TMA bulk copies: same
    distances and valid parents, single-source and host-loop."""
    off, col, roots = kron16
    g = bfs.Graph(ctx, off, col)
    if bins:
        g.set_bins(*bins)
    g.set_option(bfs.BFS_OPT_TMA_STAGE, 1)
    for r in roots[:6]:
        dist, parent, st = run_gpu(g, len(off) - 1, int(r))
        assert_parity(off, col, int(r), dist, parent, st)
    dist, parent, st = run_gpu(g, len(off) - 1, int(roots[0]), flags=bfs.BFS_HOST_LOOP)
    assert_parity(off, col, int(roots[0]), dist, parent, st)
    g.set_option(bfs.BFS_OPT_DIRECTION, 1)
    dist, parent, st = run_gpu(g, len(off) - 1, int(roots[1]))
    assert_parity(off, col, int(roots[1]), dist, parent, st)
    with pytest.raises(bfs.BfsError):
        g.set_option(bfs.BFS_OPT_TMA_STAGE, 3)
    g.close()


def test_int8_rows(ctx, kron16):
    """BFS_DIST_INT8: the same distances as int8, to device memory (aligned
    and at an odd offset, which takes the one-at-a-time conversion) and to
    host memory, with parents still int32."""
    off, col, roots = kron16
    n = len(off) - 1
    g = bfs.Graph(ctx, off, col)
    for r in roots[:4]:
        r = int(r)
        ref = oracle.bfs(off, col, r)[0]
        d8 = torch.full((n + 3,), 99, dtype=torch.int8, device="cuda")
        p = torch.empty(n, dtype=torch.int32, device="cuda")
        g.run(r, d8[:n], p)
        assert g.sync()["status"] == 0
        assert np.array_equal(d8[:n].cpu().numpy().astype(np.int32), ref)
        assert oracle.check_bfs(off, col, r, d8[:n].cpu().numpy(), p.cpu().numpy())["ok"]
        g.run(r, d8[3:])                      # 3-byte offset: not 16-byte aligned
        g.sync()
        assert np.array_equal(d8[3:].cpu().numpy().astype(np.int32), ref)
        h8 = np.full(n, 99, dtype=np.int8)
        hp = np.empty(n, dtype=np.int32)
        g.run(r, h8, hp)
        assert np.array_equal(h8.astype(np.int32), ref)
        assert oracle.check_bfs(off, col, r, h8, hp)["ok"]
    g.close()


def test_int8_rows_depth_overflow(ctx):
    """A path of 200 vertices has levels up to 199: int8 rows cannot hold
    them, and the call says so instead of wrapping."""
    off, col = G.path(200)
    g = bfs.Graph(ctx, off, col)
    h8 = np.empty(200, dtype=np.int8)
    with pytest.raises(bfs.BfsError) as e:
        g.run(0, h8)
    assert e.value.status == bfs.BFS_ERR_DEPTH_OVERFLOW
    d = np.empty(200, dtype=np.int32)
    g.run(0, d)                               # int32 rows still fine afterwards
    assert np.array_equal(d, np.arange(200, dtype=np.int32))
    g.close()
