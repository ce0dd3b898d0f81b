"""Served queries at the serving workload's sizes: the four resident
Kronecker graphs (scales 18, 20, 22 and 24, edge factor 16; the scale-22
and scale-24 graphs are the headline and batched workloads' graphs), roots
from the benchmark's pools, a burst of 128 queries followed by 128 more as
a seeded Poisson stream at 10k queries/s, submitted through bfs_submit to
the server the benchmark runs (32 GiB budget, 4 streams,
direction-optimizing graphs), each query with its own output row.  Queries
arrive while others are on the device and are packed into shared launches;
every served row must equal the oracle's distances for that query's root,
i.e. the query's result alone (Algorithm 1's d[.]).
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import graphgen
from tests import fullsize as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_13577_gb300 as bfs  # noqa: E402


def test_served_mix_every_row_equals_oracle():
    ctx = bfs.Context(0)
    graphs = []
    for spec in F.SERVE:
        off, col = F.graph(spec)
        g = bfs.Graph(ctx, off, col)
        g.set_option(bfs.BFS_OPT_DIRECTION, 1)
        pool = graphgen.pick_roots(off, 256, seed=200 + spec[1])
        graphs.append((off, col, g, pool))
    srv = bfs.Server(ctx, 32 << 30, num_streams=4)
    gids = np.array([srv.add_graph(g) for _, _, g, _ in graphs], dtype=np.int32)
    nq, rate = 256, 10_000
    rng = np.random.default_rng(rate)
    which = rng.integers(0, len(graphs), nq)
    roots = np.array([graphs[w][3][j] for w, j in zip(which, rng.integers(0, 256, nq))],
                     dtype=np.int32)
    gaps = rng.exponential(1.0 / rate, nq)
    gaps[:nq // 2] = 0.0   # a burst first: queries queue behind busy slots and share launches
    # one pinned output row per query, so every result stays for the
    # comparison and the server's result copies run asynchronously
    outs = [torch.full((len(graphs[w][0]) - 1,), -7, dtype=torch.int32).pin_memory().numpy()
            for w in which]
    tickets = []
    t0 = time.perf_counter()
    due = t0 + np.cumsum(gaps)
    for i in range(nq):
        while time.perf_counter() < due[i]:
            pass
        tickets.append(srv.submit(int(gids[which[i]]), int(roots[i]), outs[i]))
    for t in tickets:
        assert srv.wait(t, 120_000_000) == bfs.BFS_OK
        srv.release(t)
    st = srv.stats()
    srv.close()
    assert st["completed"] == nq and st["failed"] == 0
    assert st["launches"] < nq, "no two queries ever shared a launch"
    for gi, (off, col, g, _) in enumerate(graphs):
        mine = np.nonzero(which == gi)[0]
        uniq = sorted(set(int(roots[i]) for i in mine))
        ref = dict(zip(uniq, (r[0] for r in F.oracle_many(off, col, uniq))))
        for i in mine:
            assert np.array_equal(outs[i], ref[int(roots[i])]), (gi, int(roots[i]))
        g.close()
    ctx.close()
