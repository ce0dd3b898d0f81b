"""The butterfly exchange schedule (host code of the library, no GPU)
pinned to the paper's walk-through for node 0 (tests/golden/butterfly_node0.txt),
and the message count and receive-buffer bound of Section "Fanout &
Trade-offs" checked by simulating the schedule on node sets."""
from __future__ import annotations

import os

import pytest

import paper_2103_13577_gb300 as bfs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "butterfly_node0.txt")


def parse_range(t):
    out = set()
    for part in t.split(","):
        if "-" in part:
            a, b = part.split("-")
            out |= set(range(int(a), int(b) + 1))
        else:
            out.add(int(part))
    return out


def simulate(nodes, fanout):
    """holds[k] = set of nodes whose frontiers node k holds, after each round."""
    holds = [{k} for k in range(nodes)]
    history = []
    r = 0
    radix = max(2, fanout)
    rounds = 0
    p = 1
    while p < nodes:
        p *= radix
        rounds += 1
    for r in range(rounds):
        recv = [bfs.bfs_butterfly_schedule(nodes, fanout, r, k) for k in range(nodes)]
        holds = [holds[k].union(*[holds[p] for p in recv[k]]) for k in range(nodes)]
        history.append((recv, [set(h) for h in holds]))
    return history


def test_node0_walkthrough_matches_paper():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f, nodes, rnd, holds, frm = line.split()
        hist = simulate(int(nodes), int(f))
        recv, hold = hist[int(rnd)]
        assert sorted(recv[0]) == sorted(parse_range(frm)), line
        assert hold[0] == parse_range(holds), line


@pytest.mark.parametrize("nodes,fanout", [(2, 1), (8, 1), (16, 1), (64, 1), (4, 4), (16, 4),
                                          (64, 4), (64, 8), (9, 3), (27, 3)])
def test_all_nodes_learn_everything_and_message_count(nodes, fanout):
    hist = simulate(nodes, fanout)
    radix = max(2, fanout)
    assert all(h == set(range(nodes)) for h in hist[-1][1])
    messages = sum(len(p) for recv, _ in hist for p in recv)
    # each round every node receives from radix-1 others: nodes * (r-1) * log_r(nodes);
    # fanout 1 and 16 nodes: 64 messages, as the paper counts
    assert messages == nodes * (radix - 1) * len(hist)
    if (nodes, fanout) == (16, 1):
        assert messages == 64


def test_schedule_rejects_bad_rounds():
    with pytest.raises(bfs.BfsError):
        bfs.bfs_butterfly_schedule(16, 1, 4, 0)
    with pytest.raises(bfs.BfsError):
        bfs.bfs_butterfly_schedule(16, 1, 0, 16)
