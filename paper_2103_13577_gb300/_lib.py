"""ctypes declarations of include/bfs.h."""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbfs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bfs.h")

BFS_OK = 0
BFS_PENDING = 1
BFS_ERR_INVALID_ARG = -1
BFS_ERR_INVALID_GRAPH = -2
BFS_ERR_ROOT_RANGE = -3
BFS_ERR_NO_MEMORY = -4
BFS_ERR_BUDGET = -5
BFS_ERR_DEPTH_OVERFLOW = -6
BFS_ERR_TIMEOUT = -7
BFS_ERR_CUDA = -8
BFS_ERR_UNSUPPORTED = -9
BFS_ERR_CANCELLED = -10
BFS_ERR_NOT_FOUND = -11

BFS_UPLOAD_DEVICE_PTRS = 0x1
BFS_UPLOAD_NO_RELABEL = 0x2
BFS_OUT_HOST = 0x1
BFS_DIST_INT8 = 0x2
BFS_HOST_LOOP = 0x4
BFS_GRAPH_LOOP = 0x8
BFS_TUNE_BATCHED = 0x1
BFS_OPT_WARP_AGGREGATE = 1
BFS_OPT_TIMEOUT_NS = 2
BFS_OPT_CTAS_PER_SM = 3
BFS_OPT_HOT_WORDS = 4
BFS_OPT_HOT_MIN_EDGES = 5
BFS_OPT_DIRECTION = 6
BFS_OPT_DO_ALPHA = 7
BFS_OPT_DO_BETA = 8
BFS_OPT_BITMAP_FRONTIER = 9
BFS_OPT_L2_PREFETCH = 10
BFS_OPT_TMA_STAGE = 11


class BfsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("t_small", ctypes.c_int32), ("t_large", ctypes.c_int32),
                ("chunk_warp", ctypes.c_int32), ("chunk_cta", ctypes.c_int32),
                ("relabelled", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("device_bytes", ctypes.c_size_t)]


class RunStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("reached", ctypes.c_int64),
                ("edges_scanned", ctypes.c_int64), ("status", ctypes.c_int32),
                ("bottom_up_levels", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("t_small", ctypes.c_int32), ("t_large", ctypes.c_int32),
                ("chunk_warp", ctypes.c_int32), ("chunk_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("fingerprint", ctypes.c_uint64)]


class ButterflyStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("rounds_per_level", ctypes.c_int64),
                ("messages", ctypes.c_int64), ("message_entries", ctypes.c_int64),
                ("max_round_buffer_entries", ctypes.c_int64), ("max_global_queue", ctypes.c_int64),
                ("node_disagreements", ctypes.c_int64), ("nodes", ctypes.c_int32),
                ("radix", ctypes.c_int32)]


class LrbStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("kernels", ctypes.c_int64)]


class PathsStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("reached", ctypes.c_int64),
                ("edges_scanned", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("lanes", ctypes.c_int64), ("max_inflight_bytes", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t
_pp = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "bfs_context_create": (_i32, [ctypes.c_int, _vp, _sz, _pp]),
    "bfs_context_destroy": (_i32, [_vp]),
    "bfs_context_memory": (_i32, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "bfs_graph_upload": (_i32, [_vp, _vp, _vp, _i64, _i64, _u32, _vp, _pp]),
    "bfs_graph_free": (_i32, [_vp]),
    "bfs_graph_get_info": (_i32, [_vp, ctypes.POINTER(GraphInfo)]),
    "bfs_graph_set_bins": (_i32, [_vp, _i32, _i32, _i32, _i32]),
    "bfs_graph_set_option": (_i32, [_vp, _i32, _i64]),
    "bfs_run": (_i32, [_vp, _i32, _vp, _vp, _vp, _u32]),
    "bfs_graph_autotune": (_i32, [_vp, _vp, _i32, _u32, ctypes.c_char_p, ctypes.POINTER(TuneResult)]),
    "bfs_graph_sync": (_i32, [_vp, _vp, ctypes.POINTER(RunStats)]),
    "bfs_run_batch": (_i32, [_vp, _vp, _i32, _vp, _vp, _u32]),
    "bfs_run_butterfly": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, ctypes.POINTER(ButterflyStats)]),
    "bfs_run_lrb": (_i32, [_vp, _i32, _vp, _vp, ctypes.POINTER(LrbStats)]),
    "bfs_butterfly_schedule": (_i32, [_i32, _i32, _i32, _i32, ctypes.POINTER(_i32),
                                      ctypes.POINTER(_i32)]),
    "bfs_batch_sync": (_i32, [_vp, _vp, ctypes.POINTER(RunStats)]),
    "bfs_server_create": (_i32, [_vp, _sz, _i32, _pp]),
    "bfs_server_add_graph": (_i32, [_vp, _vp, ctypes.POINTER(_i32)]),
    "bfs_submit": (_i32, [_vp, _i32, _i32, _vp, ctypes.POINTER(_i64)]),
    "bfs_submit_rows": (_i32, [_vp, _i32, _i32, _vp, _u32, ctypes.POINTER(_i64)]),
    "bfs_poll": (_i32, [_vp, _i64]),
    "bfs_wait": (_i32, [_vp, _i64, _i64]),
    "bfs_release": (_i32, [_vp, _i64]),
    "bfs_ticket_times": (_i32, [_vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                ctypes.POINTER(_i64)]),
    "bfs_server_get_stats": (_i32, [_vp, ctypes.POINTER(ServerStats)]),
    "bfs_server_replay": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "bfs_server_replay_rows": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _u32, _i64, _vp, _vp,
                                      _vp]),
    "bfs_replay_single": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _vp, _vp]),
    "bfs_server_destroy": (_i32, [_vp]),
    "bfs_last_error": (ctypes.c_char_p, []),
    "bfs_status_string": (ctypes.c_char_p, [_i32]),
    "bfs_version": (_i32, []),
    "bfs_debug_set_barrier_test": (_i32, [_vp, _i32, _i64]),
    "bfs_debug_set_timeline": (_i32, [_vp, _vp, _i32]),
    "bfs_run_static": (_i32, [_vp, _vp, _i64, _i64, _i32, _vp, _vp, _vp, ctypes.POINTER(RunStats)]),
    "bfs_run_paths": (_i32, [_vp, _vp, _vp, _vp, _i64, _i64, _i32, _i32, _i32, _vp, _vp, _vp,
                             ctypes.POINTER(PathsStats)]),
}

_lib = None
_lock = threading.Lock()


def header_functions() -> list[str]:
    """Names of the functions declared in include/bfs.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfs_[a-z0-9_]+)\s*\(", text)))


def load(path: str | None = None):
    """Load libbfs.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        if path is None:
            from . import build as _build
            path = _build.build()
        if not os.path.exists(path):
            raise OSError(f"libbfs.so not found at {path}; run the package build first")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if path == LIB_PATH or _lib is None:
            _lib = L
        return L


def lib():
    return load()


def check(status: int, where: str) -> int:
    if status < 0:
        msg = load().bfs_last_error()
        raise BfsError(status, where, msg.decode() if msg else "")
    return status
