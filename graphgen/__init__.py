"""Seeded synthetic graph inputs shared by the tests and the benchmark.

Holds input generation only (no BFS arithmetic).  Graphs come back as a CSR
pair ``(off, col)``: ``off`` int64[N+1] row offsets, ``col`` int32[M] column
indices, undirected (each edge stored in both rows), rows sorted, no
self-loops and no duplicates -- the paper's input conversion (Section
"Inputs": directed inputs made undirected, duplicate and self edges removed).

Generators:
  * ``kronecker(scale, edge_factor, seed)`` -- R-MAT with initiator
    A=0.57, B=0.19, C=0.19, D=0.05, edge_factor * 2^scale generated edges,
    seeded pseudo-random vertex permutation.
  * ``erdos_renyi(scale, avg_degree, seed)`` -- avg_degree/2 * 2^scale
    uniform undirected pairs (mean directed degree ~avg_degree after cleanup).
  * ``pick_roots(off, k, seed)`` -- k distinct roots, uniform among vertices
    of degree >= 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19
KIND_RMAT, KIND_UNIFORM = 0, 1
STREAM_ROOTS = 3


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (plain gcc + OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            common = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                      ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
            lib.gg_count.argtypes = common + [i64p]
            lib.gg_count.restype = ctypes.c_int
            lib.gg_fill.argtypes = common + [i64p, i64p, i32p, i64p]
            lib.gg_fill.restype = ctypes.c_int
            lib.gg_edges_raw.argtypes = common + [i32p, i32p]
            lib.gg_edges_raw.restype = ctypes.c_int
            lib.gg_splitmix64_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_splitmix64_draw.restype = ctypes.c_uint64
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _generate(scale: int, nedges: int, a: float, b: float, c: float, seed: int, kind: int,
              permute: bool) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    n = 1 << scale
    args = (scale, nedges, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, kind, int(permute))
    deg = np.zeros(n, dtype=np.int64)
    if lib.gg_count(*args, _ptr(deg, ctypes.c_int64)) != 0:
        raise ValueError("graphgen: bad parameters")
    off_tmp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=off_tmp[1:])
    del deg
    col = np.empty(int(off_tmp[-1]) + 4, dtype=np.int32)  # +4: never zero-sized
    cursor = np.empty(n, dtype=np.int64)
    off = np.empty(n + 1, dtype=np.int64)
    rc = lib.gg_fill(*args, _ptr(off_tmp, ctypes.c_int64), _ptr(cursor, ctypes.c_int64),
                     _ptr(col, ctypes.c_int32), _ptr(off, ctypes.c_int64))
    if rc != 0:
        raise ValueError("graphgen: bad parameters")
    del cursor, off_tmp
    m = int(off[-1])
    return off, col[:m]


def kronecker(scale: int, edge_factor: int, seed: int, a: float = RMAT_A, b: float = RMAT_B,
              c: float = RMAT_C, permute: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """Undirected Kronecker (R-MAT) graph with 2^scale vertices and
    edge_factor * 2^scale generated edges, cleaned up as described above."""
    return _generate(scale, edge_factor << scale, a, b, c, seed, KIND_RMAT, permute)


def erdos_renyi(scale: int, avg_degree: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Undirected Erdos-Renyi-style graph: (avg_degree/2) * 2^scale uniform pairs."""
    return _generate(scale, (avg_degree // 2) << scale, 0.0, 0.0, 0.0, seed, KIND_UNIFORM, False)


def rmat_edges_raw(scale: int, nedges: int, seed: int, a: float = RMAT_A, b: float = RMAT_B,
                   c: float = RMAT_C, permute: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """The generated edge list before cleanup (for generator tests)."""
    lib = _load()
    src = np.empty(max(nedges, 1), dtype=np.int32)
    dst = np.empty(max(nedges, 1), dtype=np.int32)
    rc = lib.gg_edges_raw(scale, nedges, a, b, c, seed & 0xFFFFFFFFFFFFFFFF, KIND_RMAT, int(permute),
                          _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32))
    if rc != 0:
        raise ValueError("graphgen: bad parameters")
    return src[:nedges], dst[:nedges]


def splitmix64_draw(seed: int, stream: int, idx: int) -> int:
    return int(_load().gg_splitmix64_draw(seed & 0xFFFFFFFFFFFFFFFF, stream, idx))


def pick_roots(off: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k distinct roots drawn uniformly among vertices of degree >= 1."""
    n = len(off) - 1
    deg = np.diff(off)
    eligible = int(np.count_nonzero(deg))
    if k > eligible:
        raise ValueError(f"asked for {k} roots, only {eligible} vertices have degree >= 1")
    roots: list[int] = []
    seen: set[int] = set()
    i = 0
    while len(roots) < k:
        r = splitmix64_draw(seed, STREAM_ROOTS, i)
        i += 1
        v = ((r >> 32) * n) >> 32
        if deg[v] >= 1 and v not in seen:
            seen.add(v)
            roots.append(v)
    return np.asarray(roots, dtype=np.int32)


def num_threads() -> int:
    return int(_load().gg_num_threads())
