"""Pins for tests/certify.py, the PyTorch restatement of the certificate
check used on the GPU at scale 29: on the CPU it must report exactly the
counts of oracle.check_bfs (itself pinned by exhaustive enumeration) -- on
tiny graphs for every candidate distance array, and on Kronecker graphs for
the oracle's result and planted mistakes, with several chunkings."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import graphgen
import oracle
from tests.test_oracle_check_pins import TINY

torch = pytest.importorskip("torch")

from tests import certify  # noqa: E402


@pytest.fixture(autouse=True)
def _one_thread():
    # thousands of tiny tensors: thread start-up would dominate
    old = torch.get_num_threads()
    torch.set_num_threads(1)
    yield
    torch.set_num_threads(old)


def _both(off, col, root, dist, parent=None, chunk=7):
    t_off = torch.from_numpy(np.asarray(off, dtype=np.int64))
    t_col = torch.from_numpy(np.asarray(col, dtype=np.int32))
    t_d = torch.from_numpy(np.asarray(dist, dtype=np.int32))
    t_p = None if parent is None else torch.from_numpy(np.asarray(parent, dtype=np.int32))
    a = certify.check(t_off, t_col, certify.row_ranges(np.asarray(off), chunk), root, t_d, t_p)
    b = oracle.check_bfs(off, col, root, dist, parent, nthreads=2)
    return a, b


def _same(a, b):
    keys = set(certify.KINDS) | {"ok", "reached", "levels", "edges_scanned"}
    return all(a[k] == b[k] for k in keys)


@pytest.mark.parametrize("name,make,root", [TINY[1], TINY[6]], ids=[TINY[1][0], TINY[6][0]])
def test_certify_matches_checker_on_every_candidate(name, make, root):
    off, col = make()
    n = len(off) - 1
    truth = oracle.bfs(off, col, root)[0]
    for cand in itertools.product(range(-2, n), repeat=n):
        d = np.array(cand, dtype=np.int32)
        if d[root] < 0:
            continue  # levels would be undefined for an all-unreached candidate
        a, b = _both(off, col, root, d)
        assert _same(a, b), (cand, a, b)
    a, b = _both(off, col, root, truth, oracle.bfs(off, col, root)[1])
    assert a["ok"] and _same(a, b)


@pytest.mark.parametrize("chunk", [1, 1000, 1 << 30])
def test_certify_matches_checker_kronecker(chunk):
    off, col = graphgen.kronecker(12, 8, seed=3)
    rng = np.random.default_rng(4)
    for r in graphgen.pick_roots(off, 3, seed=5):
        r = int(r)
        d, p, _ = oracle.bfs(off, col, r)
        a, b = _both(off, col, r, d, p, chunk)
        assert a["ok"] and _same(a, b)
        for _ in range(8):
            d2, p2 = d.copy(), p.copy()
            v = int(rng.choice(np.nonzero(d > 0)[0]))
            k = rng.integers(0, 5)
            if k == 0:
                d2[v] += 1
            elif k == 1:
                d2[v] -= 1
            elif k == 2:
                d2[v] = -1
            elif k == 3:
                p2[v] = (p2[v] + 1) % len(d)
            else:
                d2[v] = -3
            a, b = _both(off, col, r, d2, p2, chunk)
            assert not a["ok"] and _same(a, b), (k, a, b)
