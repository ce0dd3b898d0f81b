"""Parity at the largest workload: Kronecker scale 29, edge factor 8
(536,870,912 vertices, about 8.5e9 directed entries), 64 seeded roots, in
the launch configuration the benchmark's large workload times (autotuned on
two roots).

* Every one of the 64 single-source top-down results, and 8
  direction-optimizing ones, passes the certificate check of
  tests/certify.py on the device -- the rules that hold exactly when the
  distances are the hop counts from the root -- with valid parents and the
  device's counters equal to the certificate's.
* Every lane of the 64-root batched launch with int8 rows passes the same
  check.
* On two roots the host checker (oracle.check_bfs, all host cores) reports
  the same counts as the device certificate.
* Four roots are run through the serial oracle (in parallel, one per host
  core, while the GPU work proceeds) and compared element by element.

The result to match is Algorithm 1's d[.] (Section "Preliminaries").
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import graphgen
import oracle
from tests import certify

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402

SCALE, EDGE_FACTOR, GRAPH_SEED, ROOT_SEED = 29, 8, 29, 3
ORACLE_ROOTS = 4


def test_scale29_every_root_certified():
    off, col = graphgen.kronecker(SCALE, EDGE_FACTOR, seed=GRAPH_SEED)
    n = len(off) - 1
    roots = graphgen.pick_roots(off, 64, seed=ROOT_SEED)
    pool = ThreadPoolExecutor(max_workers=ORACLE_ROOTS)
    futs = [pool.submit(oracle.bfs, off, col, int(r), None, 4096) for r in roots[:ORACLE_ROOTS]]

    ctx = bfs.Context(0)
    g = bfs.Graph(ctx, off, col)
    g.autotune(roots[:2])
    t_off = torch.from_numpy(off).cuda()
    t_col = torch.from_numpy(col).cuda()
    ranges = certify.row_ranges(off, 1 << 28)
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    kept = {}
    host_threads = max(1, (os.cpu_count() or 1) - ORACLE_ROOTS)
    for i, r in enumerate(roots):
        r = int(r)
        g.run(r, d, p)
        st = g.sync()
        res = certify.check(t_off, t_col, ranges, r, d, p)
        assert res["ok"], (r, res)
        assert (st["levels"], st["reached"], st["edges_scanned"]) == \
            (res["levels"], res["reached"], res["edges_scanned"]), r
        if i < ORACLE_ROOTS:
            kept[r] = d.cpu().numpy()
        if i < 2:
            host = oracle.check_bfs(off, col, r, kept[r], p.cpu().numpy(), nthreads=host_threads)
            assert host == {k: res[k] for k in host}, r
    g.set_option(bfs.BFS_OPT_DIRECTION, 1)
    for r in roots[:8]:
        r = int(r)
        g.run(r, d, p)
        st = g.sync()
        res = certify.check(t_off, t_col, ranges, r, d, p)
        assert res["ok"] and st["edges_scanned"] == res["edges_scanned"], (r, res)
    g.set_option(bfs.BFS_OPT_DIRECTION, 0)
    del d, p

    rows = torch.empty((64, n), dtype=torch.int8, device="cuda")
    g.run_batch(roots, rows)
    bst = g.batch_sync()
    assert bst["status"] == 0
    total_edges = 0
    for lane, r in enumerate(roots):
        res = certify.check(t_off, t_col, ranges, int(r), rows[lane])
        assert res["ok"], (lane, res)
        total_edges += res["edges_scanned"]
        if int(r) in kept:
            assert np.array_equal(rows[lane].cpu().numpy().astype(np.int32), kept[int(r)])
    assert bst["edges_scanned"] == total_edges
    del rows, t_off, t_col
    g.close()
    ctx.close()

    for r, f in zip(roots[:ORACLE_ROOTS], futs):
        d_ref, _, info = f.result()
        assert np.array_equal(kept[int(r)], d_ref), int(r)
    pool.shutdown()
