"""Per-level profiling driver: uploads a seeded Kronecker graph (edge factor
16) and runs two single-source traversals with BFS_HOST_LOOP, so that each
BFS level is its own kernel launch (one ncu result per level).

  python -m paper_2103_13577_gb300.levels_probe SCALE [hostloop|persistent|do|timeline|batch|paths]

do: host-loop launches with the direction-optimizing mode.
timeline: persistent launches with the level timeline attached; prints the
median time of init, seed and every level over 8 roots, for the L2 column
prefetch off and on, top-down and direction-optimizing.
batch: four 64-root batched launches (int32 rows, top-down, persistent) on
the roots the benchmark uses; prints the mean device time of the last two,
the frontier sums and the algorithmic bytes of one launch.
paths: two shortest-path-count traversals (bfs_run_paths, every entry kept)
on the caller's CSR copied to the device; no graph upload.
"""
from __future__ import annotations

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import graphgen
    import paper_2103_13577_gb300 as bfs

    scale = int(sys.argv[1]) if len(sys.argv) > 1 else 22
    mode = sys.argv[2] if len(sys.argv) > 2 else "hostloop"
    off, col = graphgen.kronecker(scale, 16, seed=22)
    roots = graphgen.pick_roots(off, 4, seed=3)
    ctx = bfs.Context(0)
    if mode == "paths":
        import numpy as np
        n = len(off) - 1
        d_off = torch.from_numpy(off).cuda()
        d_col = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).cuda()
        hops = torch.empty(n, dtype=torch.int32, device="cuda")
        sigma = torch.empty(n, dtype=torch.float64, device="cuda")
        for r in roots[:2]:
            print(ctx.run_paths(d_off, d_col, int(r), hops, sigma), flush=True)
        ctx.close()
        return
    g = bfs.Graph(ctx, off, col)
    n = len(off) - 1
    if mode == "batch":
        batch(bfs, g, off, graphgen.pick_roots(off, 64, seed=3))
        g.close()
        ctx.close()
        return
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    par = torch.empty(n, dtype=torch.int32, device="cuda")
    if mode == "timeline":
        timeline(bfs, g, graphgen.pick_roots(off, 8, seed=3), dist, par)
        g.close()
        ctx.close()
        return
    flags = bfs.BFS_HOST_LOOP if mode in ("hostloop", "do") else 0
    if mode == "do":
        g.set_option(bfs.BFS_OPT_DIRECTION, 1)
    for r in roots[:2]:
        g.run(int(r), dist, par, flags=flags)
        print(g.sync(), flush=True)
    g.close()
    ctx.close()


def batch(bfs, g, off, roots):
    import json

    import numpy as np
    import torch

    from paper_2103_13577_gb300 import profiling

    n = len(off) - 1
    rows = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        g.run_batch(roots, rows, stream=stream)
    g.batch_sync(stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(2):
        g.run_batch(roots, rows, stream=stream)
    ev[1].record(stream)
    st = g.batch_sync(stream)
    ms = ev[0].elapsed_time(ev[1]) / 2
    deg = torch.from_numpy(np.diff(off)).cuda()
    sizes, degs, reached = profiling.batch_frontier_sums(rows, deg)
    b = profiling.batch_algorithmic_bytes(sizes, degs, reached, n, len(roots), 4)
    print(json.dumps({"ms": ms, "levels": int(st["levels"]), "edges_scanned": int(st["edges_scanned"]),
                      "frontier_entries": sizes, "frontier_edges": degs, "reached": reached,
                      "algorithmic_bytes": b, "gbs": b / (ms * 1e-3) / 1e9}), flush=True)


def timeline(bfs, g, roots, dist, par):
    import numpy as np
    import torch

    stamps = torch.zeros(64, dtype=torch.int64, device="cuda")
    bfs.bfs_debug_set_timeline(g.handle, stamps)
    for direction in (0, 1):
        g.set_option(bfs.BFS_OPT_DIRECTION, direction)
        for pf in (0, 1):
            g.set_option(bfs.BFS_OPT_L2_PREFETCH, pf)
            rows = []
            for rep in range(2):
                for r in roots:
                    stamps.zero_()
                    g.run(int(r), dist, par)
                    st = g.sync()
                    t = stamps.cpu().numpy()
                    k = 3 + st["levels"]
                    if rep == 1:
                        rows.append(np.diff(t[:k]) / 1e3)
            width = max(len(x) for x in rows)
            a = np.full((len(rows), width), np.nan)
            for i, x in enumerate(rows):
                a[i, :len(x)] = x
            med = np.nanmedian(a, axis=0)
            tot = np.median([x.sum() for x in rows])
            names = ["init", "seed"] + [f"L{i}" for i in range(width - 2)]
            print(f"direction {direction} prefetch {pf} total_us {tot:.1f} " +
                  " ".join(f"{nm}={v:.1f}" for nm, v in zip(names, med)), flush=True)
    bfs.bfs_debug_set_timeline(g.handle, None)


if __name__ == "__main__":
    main()
