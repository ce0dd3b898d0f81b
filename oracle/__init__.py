"""CPU oracle for breadth-first search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The GPU library never calls it and shares no
code with it (the only common module is ``graphgen``, which makes inputs).

* ``bfs(off, col, root)`` -- serial FIFO-queue BFS (Algorithm 1 run on one
  thread; ``bfs_oracle.c``).  Returns int32 ``dist`` (-1 = unreachable,
  Section "Preliminaries": d = infinity), one valid int32 ``parent``, and
  an info dict (levels, per-level vertex counts, scanned entries m_c).
* ``bfs_multi(off, col, roots)`` -- one independent BFS per root, k x n.
* ``bfs_paths(off, col, root, weight, lo, hi)`` -- shortest-path counts
  (Brandes' forward phase) on the entries whose weight lies in [lo, hi]
  (all entries when ``weight`` is None): int32 ``hops``, float64 ``sigma``.
* ``check_tree(off, col, root, dist, parent)`` -- Graph500-style checks of a
  BFS result that do not depend on which of several valid parents was
  chosen (used to accept GPU parents).
* ``check_bfs(off, col, root, dist, parent=None)`` -- the same rules in
  directed form plus a predecessor witness per reached vertex, streamed over
  the CSR on all host cores (``bfs_check.c``): holds exactly when ``dist``
  is the shortest-path hop count from ``root`` (and, with ``parent``, when
  the parents form a valid BFS tree); used where the serial oracle is too
  slow to run on every root (scale 29).

Pins: ``tests/test_oracle_pins.py`` checks this oracle against Floyd-Warshall
brute force, closed-form distances, scipy's breadth-first search, and
union-find components; ``tests/test_oracle_paths_pins.py`` checks the path
counts against walk counts from adjacency-matrix powers and closed forms;
``tests/test_oracle_check_pins.py`` checks ``check_bfs`` by exhaustive
enumeration of candidate distance and parent arrays on tiny graphs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_CHECK_SRC = os.path.join(_HERE, "bfs_check.c")
_CHECK_PATH = os.path.join(_HERE, "libbfscheck.so")
_lib = None
_check_lib = None
_lock = threading.Lock()


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the oracle with plain gcc (no OpenMP, no vectorisation flags),
    and the invariant checker (plain gcc with POSIX threads)."""
    if src is None and out is None:
        build_check(force)
    src = src or _SRC
    out = out or _LIB_PATH
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def build_check(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    src = src or _CHECK_SRC
    out = out or _CHECK_PATH
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-pthread", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def load_check(path: str | None = None):
    """Load the invariant checker (the default build, or another compiled copy)."""
    global _check_lib

    def bind(lib):
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_check_bfs.argtypes = [ctypes.c_int64, i64p, i32p, ctypes.c_int64, i32p, i32p,
                                         ctypes.c_int32, i64p, i64p, i64p, i64p]
        lib.oracle_check_bfs.restype = ctypes.c_int64
        return lib

    if path is None:
        with _lock:
            if _check_lib is None:
                _check_lib = bind(ctypes.CDLL(build_check()))
        return _check_lib
    return bind(ctypes.CDLL(path))


def load(path: str | None = None):
    """Load the oracle library (the default build, or another compiled copy)."""
    global _lib
    if path is None:
        with _lock:
            if _lib is None:
                _lib = _bind(ctypes.CDLL(build()))
        return _lib
    return _bind(ctypes.CDLL(path))


def _bind(lib):
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_bfs.argtypes = [ctypes.c_int64, i64p, i32p, ctypes.c_int64, i32p, i32p, i64p,
                               ctypes.c_int64, i64p]
    lib.oracle_bfs.restype = ctypes.c_int64
    lib.oracle_bfs_multi.argtypes = [ctypes.c_int64, i64p, i32p, i64p, ctypes.c_int64, i32p, i64p]
    lib.oracle_bfs_multi.restype = ctypes.c_int64
    lib.oracle_bfs_paths.argtypes = [ctypes.c_int64, i64p, i32p, i32p, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int64, i32p,
                                     ctypes.POINTER(ctypes.c_double), i64p]
    lib.oracle_bfs_paths.restype = ctypes.c_int64
    return lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _csr(off, col):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return off, col


def bfs(off, col, root, lib=None, max_levels=None):
    """Serial BFS from ``root``: (dist int32[n], parent int32[n], info).
    ``max_levels`` bounds the per-level counts kept in ``info`` (default: as
    many as the graph can have levels)."""
    lib = lib or load()
    off, col = _csr(off, col)
    n = len(off) - 1
    if not (0 <= root < n):
        raise ValueError("root out of range")
    dist = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    max_levels = n + 1 if max_levels is None else int(max_levels)
    levels = np.zeros(max_levels, dtype=np.int64)
    scanned = np.zeros(1, dtype=np.int64)
    nl = lib.oracle_bfs(n, _p(off, ctypes.c_int64), _p(col, ctypes.c_int32), int(root),
                        _p(dist, ctypes.c_int32), _p(parent, ctypes.c_int32),
                        _p(levels, ctypes.c_int64), max_levels, _p(scanned, ctypes.c_int64))
    if nl < 0:
        raise RuntimeError(f"oracle_bfs failed ({nl})")
    info = {"levels": int(nl), "level_sizes": levels[:min(nl, max_levels)].copy(),
            "edges_scanned": int(scanned[0]),
            "reached": int(np.count_nonzero(dist >= 0))}
    return dist, parent, info


def bfs_multi(off, col, roots, lib=None):
    """One independent BFS per root: (dist int32[k][n], scanned int64[k])."""
    lib = lib or load()
    off, col = _csr(off, col)
    n = len(off) - 1
    roots = np.ascontiguousarray(roots, dtype=np.int64)
    k = len(roots)
    dist = np.empty((k, n), dtype=np.int32)
    scanned = np.zeros(max(k, 1), dtype=np.int64)
    rc = lib.oracle_bfs_multi(n, _p(off, ctypes.c_int64), _p(col, ctypes.c_int32),
                              _p(roots, ctypes.c_int64), k, _p(dist, ctypes.c_int32),
                              _p(scanned, ctypes.c_int64))
    if rc < 0:
        raise RuntimeError(f"oracle_bfs_multi failed ({rc})")
    return dist, scanned[:k]


def bfs_paths(off, col, root, weight=None, lo=0, hi=0, lib=None):
    """Shortest-path counts from ``root`` over the entries e with
    lo <= weight[e] <= hi (every entry when ``weight`` is None):
    (hops int32[n], sigma float64[n], info)."""
    lib = lib or load()
    off, col = _csr(off, col)
    n = len(off) - 1
    if not (0 <= root < n):
        raise ValueError("root out of range")
    wp = None
    if weight is not None:
        weight = np.ascontiguousarray(weight, dtype=np.int32)
        if len(weight) < off[-1]:
            raise ValueError("weight shorter than the column array")
        if weight.size == 0:
            weight = np.zeros(1, dtype=np.int32)
        wp = _p(weight, ctypes.c_int32)
    hops = np.empty(n, dtype=np.int32)
    sigma = np.empty(n, dtype=np.float64)
    scanned = np.zeros(1, dtype=np.int64)
    nl = lib.oracle_bfs_paths(n, _p(off, ctypes.c_int64), _p(col, ctypes.c_int32), wp, int(lo),
                              int(hi), int(root), _p(hops, ctypes.c_int32),
                              _p(sigma, ctypes.c_double), _p(scanned, ctypes.c_int64))
    if nl < 0:
        raise RuntimeError(f"oracle_bfs_paths failed ({nl})")
    info = {"levels": int(nl), "edges_scanned": int(scanned[0]),
            "reached": int(np.count_nonzero(hops >= 0))}
    return hops, sigma, info


def check_tree(off, col, root, dist, parent, undirected=True):
    """Graph500-style validation of a BFS result; returns a list of problems
    (empty when valid).  Checks: dist[root] = 0 and parent[root] = root; every
    reached v != root has a parent p with an edge p -> v and dist[p] =
    dist[v] - 1 (so following parents reaches the root in dist[v] steps);
    unreached vertices have parent -1; on undirected graphs every edge joins
    two reached or two unreached vertices and |dist[u] - dist[v]| <= 1."""
    off = np.asarray(off, dtype=np.int64)
    col = np.asarray(col, dtype=np.int32)
    dist = np.asarray(dist, dtype=np.int64)
    parent = np.asarray(parent, dtype=np.int64)
    n = len(off) - 1
    bad = []
    if dist[root] != 0:
        bad.append("dist[root] != 0")
    if parent[root] != root:
        bad.append("parent[root] != root")
    reached = dist >= 0
    unreached_with_parent = np.nonzero(~reached & (parent != -1))[0]
    if unreached_with_parent.size:
        bad.append(f"{unreached_with_parent.size} unreached vertices have a parent")
    others = np.nonzero(reached)[0]
    others = others[others != root]
    if others.size:
        p = parent[others]
        if np.any((p < 0) | (p >= n)):
            bad.append("reached vertex with parent out of range")
            return bad
        if np.any(dist[p] != dist[others] - 1):
            bad.append("parent not one level closer to the root")
        # edge p -> v must exist: binary search in p's sorted-or-not row
        src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
        key_edges = src * n + col.astype(np.int64)
        key_edges.sort()
        key_par = p * n + others
        pos = np.searchsorted(key_edges, key_par)
        pos = np.minimum(pos, max(len(key_edges) - 1, 0))
        if len(key_edges) == 0 or np.any(key_edges[pos] != key_par):
            bad.append("parent is not adjacent to the vertex")
    if undirected and len(col):
        src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
        du, dv = dist[src], dist[col]
        if np.any((du >= 0) != (dv >= 0)):
            bad.append("edge between reached and unreached vertex")
        both = (du >= 0) & (dv >= 0)
        if np.any(np.abs(du[both] - dv[both]) > 1):
            bad.append("edge spans more than one level")
    return bad


CHECK_KINDS = ("root_dist", "below_minus_one", "reach_gap", "level_skip", "no_witness",
               "root_parent", "unreached_parent", "bad_parent")


def check_bfs(off, col, root, dist, parent=None, nthreads=None, lib=None):
    """Certificate check of a BFS result (``bfs_check.c``): dist (int32 or
    int8, -1 unreached) equals the hop distances from ``root`` exactly when
    every count is zero; with ``parent`` the tree is checked too.  Returns a
    dict: ``ok``, the violation count of each kind (``CHECK_KINDS``),
    ``reached``, ``levels`` and ``edges_scanned`` (entries of the reached
    rows).  The CSR itself must be valid (columns in [0, n))."""
    lib = lib or load_check()
    off, col = _csr(off, col)
    n = len(off) - 1
    if not (0 <= root < n):
        raise ValueError("root out of range")
    dist = np.ascontiguousarray(dist, dtype=np.int32)
    if len(dist) != n:
        raise ValueError("dist has the wrong length")
    pp = None
    if parent is not None:
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        if len(parent) != n:
            raise ValueError("parent has the wrong length")
        pp = _p(parent, ctypes.c_int32)
    bad = np.zeros(len(CHECK_KINDS), dtype=np.int64)
    out = np.zeros(3, dtype=np.int64)
    nt = int(nthreads or os.cpu_count() or 1)
    rc = lib.oracle_check_bfs(n, _p(off, ctypes.c_int64), _p(col, ctypes.c_int32), int(root),
                              _p(dist, ctypes.c_int32), pp, nt, _p(bad, ctypes.c_int64),
                              _p(out[0:], ctypes.c_int64), _p(out[1:], ctypes.c_int64),
                              _p(out[2:], ctypes.c_int64))
    if rc < 0:
        raise RuntimeError(f"oracle_check_bfs failed ({rc})")
    res = {k: int(v) for k, v in zip(CHECK_KINDS, bad)}
    res.update(ok=bool(rc == 0), reached=int(out[0]), levels=int(out[1]),
               edges_scanned=int(out[2]))
    return res
