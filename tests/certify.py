"""The certificate check of oracle/bfs_check.c restated with plain PyTorch
ops, for results too large to bring to the host for every root (scale 29:
8.5e9 entries).  Test infrastructure: it uses torch's own gather, compare
and scatter kernels, none of the library's.

For a root r and distances d (-1 unreached) on a CSR (off, col) held as
torch tensors on the device, the rules are those of bfs_check.c:
  C0 d[r] = 0;  C1 no d below -1;
  C2 an entry u -> v out of a reached u leads to a reached v;
  C3 along it d[v] <= d[u] + 1;
  C4 every reached v != r has an entry u -> v with u reached and d[u] = d[v] - 1;
and with parents p: P0 p[r] = r; P1 unreached -> -1; P2 a reached v != r
has an entry p[v] -> v with p[v] reached and d[p[v]] = d[v] - 1.
Together C0-C4 hold exactly when d equals the hop distances from r.  The
entries are processed in row ranges of about `chunk` entries; counts come
back by kind, as oracle.check_bfs reports them.
"""
from __future__ import annotations

import torch

KINDS = ("root_dist", "below_minus_one", "reach_gap", "level_skip", "no_witness",
         "root_parent", "unreached_parent", "bad_parent")


def row_ranges(off_host, chunk):
    """[v0, v1) row ranges of about `chunk` entries each (off_host: numpy)."""
    import numpy as np
    n = len(off_host) - 1
    bounds = np.searchsorted(off_host, np.arange(0, off_host[-1] + chunk, chunk), side="left")
    bounds = np.unique(np.concatenate([[0], np.minimum(bounds, n), [n]]))
    return [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


@torch.no_grad()
def check(off, col, ranges, root, dist, parent=None):
    """off: int64[n+1], col: int32[nnz], dist: int32/int8[n], parent:
    int32[n] or None -- torch tensors on one device.  ranges: row_ranges()."""
    dev = dist.device
    n = dist.numel()
    d = dist.to(torch.int32)
    bad = dict.fromkeys(KINDS, 0)
    witness = torch.zeros(n, dtype=torch.bool, device=dev)
    mark = torch.zeros(n, dtype=torch.bool, device=dev) if parent is not None else None
    scanned = 0
    for v0, v1 in ranges:
        e0, e1 = int(off[v0].item()), int(off[v1].item())
        if e1 == e0:
            continue
        deg = off[v0 + 1:v1 + 1] - off[v0:v1]
        du_rows = d[v0:v1]
        scanned += int(deg[du_rows >= 0].sum().item())
        u = torch.repeat_interleave(torch.arange(v0, v1, device=dev, dtype=torch.int32), deg,
                                    output_size=e1 - e0)
        du = du_rows.repeat_interleave(deg, output_size=e1 - e0)
        tgt = col[e0:e1].long()
        dv = d[tgt]
        reached_u = du >= 0
        bad["reach_gap"] += int((reached_u & (dv < 0)).sum().item())
        bad["level_skip"] += int((reached_u & (dv > du + 1)).sum().item())
        step = reached_u & (dv == du + 1)
        witness[tgt[step]] = True
        if parent is not None:
            hit = step & (parent[tgt] == u)
            mark[tgt[hit]] = True
        del u, du, tgt, dv, reached_u, step
    reached = d >= 0
    others = reached.clone()
    others[root] = False
    bad["below_minus_one"] = int((d < -1).sum().item())
    bad["no_witness"] = int((others & ~witness).sum().item())
    bad["root_dist"] = int(d[root].item() != 0)
    if parent is not None:
        bad["root_parent"] = int(parent[root].item() != root)
        bad["unreached_parent"] = int(((d == -1) & (parent != -1)).sum().item())
        bad["bad_parent"] = int((others & ~mark).sum().item())
    out = dict(bad)
    out.update(ok=sum(bad.values()) == 0, reached=int(reached.sum().item()),
               levels=int(d.max().item()) + 1, edges_scanned=scanned)
    return out
