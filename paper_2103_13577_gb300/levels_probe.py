"""Per-level profiling driver: uploads a seeded Kronecker graph (edge factor
16) and runs two single-source traversals with BFS_HOST_LOOP, so that each
BFS level is its own kernel launch (one ncu result per level).

  python -m paper_2103_13577_gb300.levels_probe SCALE [hostloop|persistent|do]

do: host-loop launches with the direction-optimizing mode.
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
    g = bfs.Graph(ctx, off, col)
    n = len(off) - 1
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    par = torch.empty(n, dtype=torch.int32, device="cuda")
    flags = bfs.BFS_HOST_LOOP if mode in ("hostloop", "do") else 0
    if mode == "do":
        g.set_option(bfs.BFS_OPT_DIRECTION, 1)
    for r in roots[:2]:
        g.run(int(r), dist, par, flags=flags)
        print(g.sync(), flush=True)
    g.close()
    ctx.close()


if __name__ == "__main__":
    main()
