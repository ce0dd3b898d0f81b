"""Parity at the benchmark sizes, on every root, in the launch
configurations the benchmark times.

* Kronecker scale 22, edge factor 16, the headline graph and its 64 roots:
  every root single-source top-down (the persistent kernel the headline
  times), direction-optimizing, CUDA-graph loop and the paper's LRB scheme,
  plus the 64-root batched launch on the same graph (top-down and
  direction-optimizing) -- every distance array equal to the oracle's
  element by element, parents valid by the certificate check, and the
  device's counters (levels, reached, m_c) equal to the oracle's.
* The scale-24 batched workload on the Kronecker graph and the Erdos-Renyi
  graph (2^24 vertices, average degree 32), autotuned as the benchmark does:
  the 64 single-source runs (top-down and direction-optimizing) and every
  lane of the 64-root launches with int32 and int8 rows, top-down and
  direction-optimizing, against the oracle row of that lane's root.

The result to match is Algorithm 1's d[.] (Section "Preliminaries": level k
holds the vertices at distance k).
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import certify
from tests import fullsize as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = bfs.Context(0)
    yield c
    c.close()


class DeviceCsr:
    """The caller's CSR on the device for tests/certify.py."""

    def __init__(self, off, col):
        self.off = torch.from_numpy(off).cuda()
        self.col = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).cuda()
        self.ranges = certify.row_ranges(off, 1 << 26)


def _single_source_all_roots(g, off, col, roots, ref, flags=0, lrb=False, dev_csr=None):
    """Every root: distances equal to the oracle's; parents and counters by
    the certificate check -- on the host (oracle.check_bfs) or, given
    dev_csr, with tests/certify.py on the device."""
    n = len(off) - 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    for i, r in enumerate(roots):
        r = int(r)
        d_ref, _, info = ref[i]
        if lrb:
            g.run_lrb(r, d)
            assert np.array_equal(d.cpu().numpy(), d_ref), ("lrb", r)
            continue
        g.run(r, d, p, flags=flags)
        st = g.sync()
        dist = d.cpu().numpy()
        assert np.array_equal(dist, d_ref), (r, flags)
        if dev_csr is None:
            chk = oracle.check_bfs(off, col, r, dist, p.cpu().numpy())
        else:
            chk = certify.check(dev_csr.off, dev_csr.col, dev_csr.ranges, r, d, p)
        assert chk["ok"], (r, chk)
        assert chk["edges_scanned"] == info["edges_scanned"]
        assert (st["levels"], st["reached"], st["edges_scanned"]) == \
            (info["levels"], info["reached"], info["edges_scanned"]), r


def _batched_all_lanes(g, roots, ref, n, dtype):
    rows = torch.empty((len(roots), n), dtype=dtype, device="cuda")
    g.run_batch(roots, rows)
    st = g.batch_sync()
    assert st["status"] == 0
    host = rows.cpu().numpy()
    for lane in range(len(roots)):
        assert np.array_equal(host[lane].astype(np.int32), ref[lane][0]), (dtype, lane)
    assert st["edges_scanned"] == sum(r[2]["edges_scanned"] for r in ref)
    assert st["reached"] == sum(r[2]["reached"] for r in ref)
    assert st["levels"] == max(r[2]["levels"] for r in ref)
    del rows


def test_scale22_every_root_every_mode(ctx):
    off, col = F.graph(F.KRON_S22)
    roots = graphgen.pick_roots(off, 64, seed=F.ROOT_SEED)
    ref = F.oracle_many(off, col, roots)
    g = bfs.Graph(ctx, off, col)
    _single_source_all_roots(g, off, col, roots, ref)
    _single_source_all_roots(g, off, col, roots, ref, lrb=True)
    g.set_option(bfs.BFS_OPT_DIRECTION, 1)
    _single_source_all_roots(g, off, col, roots, ref)
    g.set_option(bfs.BFS_OPT_DIRECTION, 0)
    _single_source_all_roots(g, off, col, roots[:16], ref[:16], flags=bfs.BFS_GRAPH_LOOP)
    n = len(off) - 1
    for direction in (0, 1):
        g.set_option(bfs.BFS_OPT_DIRECTION, direction)
        _batched_all_lanes(g, roots, ref, n, torch.int32)
    g.set_option(bfs.BFS_OPT_DIRECTION, 0)
    # the device-side certificate used at larger sizes reports what the host
    # checker reports, on the GPU's own results and on a planted bad parent
    dev_csr = DeviceCsr(off, col)
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots[:3]:
        r = int(r)
        g.run(r, d, p)
        g.sync()
        host = oracle.check_bfs(off, col, r, d.cpu().numpy(), p.cpu().numpy())
        dev = certify.check(dev_csr.off, dev_csr.col, dev_csr.ranges, r, d, p)
        assert host == {k: dev[k] for k in host}
        v = int(torch.nonzero(d == 2)[0].item())
        p[v] = r
        host = oracle.check_bfs(off, col, r, d.cpu().numpy(), p.cpu().numpy())
        dev = certify.check(dev_csr.off, dev_csr.col, dev_csr.ranges, r, d, p)
        assert not host["ok"] and host == {k: dev[k] for k in host}
    g.close()


@pytest.mark.parametrize("spec", [F.KRON_S24, F.ER_S24], ids=["kronecker", "erdos_renyi"])
def test_scale24_batched_every_lane(ctx, spec):
    off, col = F.graph(spec)
    n = len(off) - 1
    roots = graphgen.pick_roots(off, 64, seed=F.ROOT_SEED)
    ref = F.oracle_many(off, col, roots)
    g = bfs.Graph(ctx, off, col)
    dev_csr = DeviceCsr(off, col)
    # the benchmark's launch configuration: single-source runs tuned on four
    # roots, batched launches tuned on all 64
    g.autotune(roots[:4])
    for direction in (0, 1):
        g.set_option(bfs.BFS_OPT_DIRECTION, direction)
        _single_source_all_roots(g, off, col, roots, ref, dev_csr=dev_csr)
    g.set_option(bfs.BFS_OPT_DIRECTION, 0)
    g.autotune(roots, batched=True)
    for direction in (0, 1):
        g.set_option(bfs.BFS_OPT_DIRECTION, direction)
        for dtype in (torch.int32, torch.int8):
            _batched_all_lanes(g, roots, ref, n, dtype)
    g.close()
    del dev_csr
