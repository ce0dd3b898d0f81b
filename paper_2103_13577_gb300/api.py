"""Argument marshalling for the C ABI (include/bfs.h).

Functions carry the C names.  Buffers may be numpy arrays (host memory) or
torch CUDA tensors (device memory); the ``BFS_OUT_HOST`` /
``BFS_UPLOAD_DEVICE_PTRS`` flags follow from which kind is passed.  Streams
may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None
(torch's current stream when torch has initialised CUDA, else the legacy
default stream).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (BFS_DIST_INT8, BFS_OUT_HOST, BFS_TUNE_BATCHED, BFS_UPLOAD_DEVICE_PTRS,
                   ButterflyStats, GraphInfo, LrbStats, PathsStats, RunStats, ServerStats,
                   TuneResult, check)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _buf(x, dtype: np.dtype | None = None):
    """(pointer, is_device) of a numpy array or torch tensor."""
    if x is None:
        return None, False
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {x.dtype}")
        return x.ctypes.data, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None:
            want = {np.dtype(np.int32): "torch.int32", np.dtype(np.int64): "torch.int64",
                    np.dtype(np.int8): "torch.int8", np.dtype(np.uint8): "torch.uint8",
                    np.dtype(np.float64): "torch.float64"}[np.dtype(dtype)]
            if str(x.dtype) != want:
                raise TypeError(f"expected {want}, got {x.dtype}")
        return x.data_ptr(), x.is_cuda
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------- functions

def bfs_context_create(device: int = 0, arena=None) -> int:
    ptr = ctypes.c_void_p()
    a, nbytes = None, 0
    if arena is not None:
        a, is_dev = _buf(arena)
        if not is_dev:
            raise ValueError("arena must be device memory")
        nbytes = arena.numel() * arena.element_size()
    check(_lib.lib().bfs_context_create(device, a, nbytes, ctypes.byref(ptr)), "bfs_context_create")
    return ptr.value


def bfs_context_destroy(ctx: int) -> None:
    check(_lib.lib().bfs_context_destroy(ctx), "bfs_context_destroy")


def bfs_graph_upload(ctx: int, row_off, col, flags: int = 0, stream=None) -> int:
    p_off, dev_off = _buf(row_off, np.int64)
    p_col, dev_col = _buf(col, np.int32)
    if dev_off != dev_col:
        raise ValueError("row_off and col must both be host or both be device buffers")
    if dev_off:
        flags |= BFS_UPLOAD_DEVICE_PTRS
    n = (row_off.shape[0] if hasattr(row_off, "shape") else len(row_off)) - 1
    nnz = col.shape[0] if hasattr(col, "shape") else len(col)
    out = ctypes.c_void_p()
    check(_lib.lib().bfs_graph_upload(ctx, p_off, p_col if nnz else None, n, nnz, flags,
                                      _stream(stream), ctypes.byref(out)), "bfs_graph_upload")
    return out.value


def bfs_graph_free(g: int) -> None:
    check(_lib.lib().bfs_graph_free(g), "bfs_graph_free")


def bfs_graph_get_info(g: int) -> dict:
    info = GraphInfo()
    check(_lib.lib().bfs_graph_get_info(g, ctypes.byref(info)), "bfs_graph_get_info")
    return {f: getattr(info, f) for f, _ in GraphInfo._fields_}


def bfs_graph_set_bins(g: int, t_small: int, t_large: int, chunk_warp: int, chunk_cta: int) -> None:
    check(_lib.lib().bfs_graph_set_bins(g, t_small, t_large, chunk_warp, chunk_cta),
          "bfs_graph_set_bins")


def bfs_graph_set_option(g: int, option: int, value: int) -> None:
    check(_lib.lib().bfs_graph_set_option(g, option, int(value)), "bfs_graph_set_option")


def bfs_graph_autotune(g: int, roots, batched: bool = False, cache_path: str | None = None) -> dict:
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    res = TuneResult()
    check(_lib.lib().bfs_graph_autotune(g, roots.ctypes.data, len(roots),
                                        BFS_TUNE_BATCHED if batched else 0,
                                        cache_path.encode() if cache_path else None,
                                        ctypes.byref(res)), "bfs_graph_autotune")
    return {f: getattr(res, f) for f, _ in TuneResult._fields_}


def bfs_run(g: int, root: int, dist, parent=None, stream=None, flags: int = 0) -> None:
    flags |= _row_flags(dist)
    p_dist, dev = _buf(dist)
    p_par, dev_p = _buf(parent, np.int32)
    if parent is not None and dev_p != dev:
        raise ValueError("dist and parent must both be host or both be device buffers")
    if not dev:
        flags |= BFS_OUT_HOST
    check(_lib.lib().bfs_run(g, int(root), p_dist, p_par, _stream(stream), flags), "bfs_run")


def bfs_run_static(row_off, col, root: int, dist, parent=None, stream=None,
                   wait: bool = True) -> dict | None:
    """Single-source traversal on a CSR already on the device, using the
    library's fixed scratch (no device allocation).  Returns the traversal
    statistics when wait is True."""
    p_off, d_off = _buf(row_off, np.int64)
    p_col, d_col = _buf(col, np.int32)
    p_dist, d_dist = _buf(dist, np.int32)
    p_par, d_par = _buf(parent, np.int32)
    if not (d_off and d_col and d_dist and (parent is None or d_par)):
        raise ValueError("bfs_run_static takes device buffers only")
    n = row_off.shape[0] - 1
    nnz = col.shape[0]
    st = RunStats()
    check(_lib.lib().bfs_run_static(p_off, p_col if nnz else None, n, nnz, int(root), p_dist, p_par,
                                    _stream(stream), ctypes.byref(st) if wait else None),
          "bfs_run_static")
    return {f: getattr(st, f) for f, _ in RunStats._fields_} if wait else None


def bfs_run_butterfly(g: int, root: int, nodes: int, fanout: int, dist, stream=None) -> dict:
    """Algorithm 2 emulated with `nodes` virtual compute nodes on this GPU."""
    p_dist, dev = _buf(dist, np.int32)
    if not dev:
        raise ValueError("dist must be a device buffer")
    st = ButterflyStats()
    check(_lib.lib().bfs_run_butterfly(g, int(root), nodes, fanout, p_dist, _stream(stream),
                                       ctypes.byref(st)), "bfs_run_butterfly")
    return {f: getattr(st, f) for f, _ in ButterflyStats._fields_}


def bfs_run_lrb(g: int, root: int, dist, stream=None) -> dict:
    """The paper's per-bin-kernel traversal (comparison path)."""
    p_dist, dev = _buf(dist, np.int32)
    if not dev:
        raise ValueError("dist must be a device buffer")
    st = LrbStats()
    check(_lib.lib().bfs_run_lrb(g, int(root), p_dist, _stream(stream), ctypes.byref(st)),
          "bfs_run_lrb")
    return {f: getattr(st, f) for f, _ in LrbStats._fields_}


def bfs_run_paths(ctx: int, row_off, col, root: int, hops, sigma, weight=None, lo: int = 0,
                  hi: int = 0, stream=None) -> dict:
    """Shortest-path counts (hops int32, sigma float64) from `root` over the
    entries e of a device CSR with lo <= weight[e] <= hi (every entry when
    weight is None).  Device buffers only; returns the traversal
    statistics."""
    p_off, d_off = _buf(row_off, np.int64)
    p_col, d_col = _buf(col, np.int32)
    p_w, d_w = _buf(weight, np.int32)
    p_h, d_h = _buf(hops, np.int32)
    p_s, d_s = _buf(sigma, np.float64)
    if not (d_off and d_col and d_h and d_s and (weight is None or d_w)):
        raise ValueError("bfs_run_paths takes device buffers only")
    n = row_off.shape[0] - 1
    nnz = col.shape[0]
    st = PathsStats()
    check(_lib.lib().bfs_run_paths(ctx, p_off, p_col if nnz else None, p_w, n, nnz, int(lo),
                                   int(hi), int(root), p_h, p_s, _stream(stream),
                                   ctypes.byref(st)), "bfs_run_paths")
    return {f: getattr(st, f) for f, _ in PathsStats._fields_}


def bfs_butterfly_schedule(nodes: int, fanout: int, round_: int, node: int) -> list[int]:
    """Nodes whose global queues `node` receives in round `round_` (host only)."""
    buf = (ctypes.c_int32 * 16)()
    cnt = ctypes.c_int32()
    check(_lib.lib().bfs_butterfly_schedule(nodes, fanout, round_, node, buf, ctypes.byref(cnt)),
          "bfs_butterfly_schedule")
    return [buf[i] for i in range(cnt.value)]


def bfs_debug_set_timeline(g: int, stamps) -> None:
    """Attach a device int64 tensor (>= 3 entries) that every persistent
    traversal fills with %globaltimer stamps: [0] start, [1] after init, [2]
    after the seed; single-source [3 + L] after level L, batched [3 + 2L]
    after level L's expansion and [4 + 2L] after its sweep.  None detaches."""
    if stamps is None:
        check(_lib.lib().bfs_debug_set_timeline(g, None, 0), "bfs_debug_set_timeline")
        return
    p, dev = _buf(stamps, np.int64)
    if not dev:
        raise ValueError("the timeline must be a device tensor")
    check(_lib.lib().bfs_debug_set_timeline(g, p, int(stamps.numel())), "bfs_debug_set_timeline")


def bfs_graph_sync(g: int, stream=None) -> dict:
    st = RunStats()
    check(_lib.lib().bfs_graph_sync(g, _stream(stream), ctypes.byref(st)), "bfs_graph_sync")
    return {f: getattr(st, f) for f, _ in RunStats._fields_}


def bfs_run_batch(g: int, roots, dist, stream=None, flags: int = 0) -> None:
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    p_dist, dev = _buf(dist)
    dt = dist.dtype if isinstance(dist, np.ndarray) else str(dist.dtype)
    if str(dt) in ("int8", "torch.int8"):
        flags |= BFS_DIST_INT8
    elif str(dt) not in ("int32", "torch.int32"):
        raise TypeError("dist must be int32 or int8")
    if not dev:
        flags |= BFS_OUT_HOST
    check(_lib.lib().bfs_run_batch(g, roots.ctypes.data, len(roots), p_dist, _stream(stream), flags),
          "bfs_run_batch")


def bfs_batch_sync(g: int, stream=None) -> dict:
    st = RunStats()
    check(_lib.lib().bfs_batch_sync(g, _stream(stream), ctypes.byref(st)), "bfs_batch_sync")
    return {f: getattr(st, f) for f, _ in RunStats._fields_}


def bfs_server_create(ctx: int, memory_budget: int, num_streams: int = 4) -> int:
    out = ctypes.c_void_p()
    check(_lib.lib().bfs_server_create(ctx, memory_budget, num_streams, ctypes.byref(out)),
          "bfs_server_create")
    return out.value


def bfs_server_add_graph(s: int, g: int) -> int:
    gid = ctypes.c_int32()
    check(_lib.lib().bfs_server_add_graph(s, g, ctypes.byref(gid)), "bfs_server_add_graph")
    return gid.value


def _row_flags(buf) -> int:
    """BFS_DIST_INT8 for int8 rows, 0 for int32 rows (numpy or torch)."""
    dt = str(buf.dtype)
    if dt in ("int8", "torch.int8"):
        return BFS_DIST_INT8
    if dt not in ("int32", "torch.int32"):
        raise TypeError("rows must be int32 or int8")
    return 0


def bfs_submit(s: int, graph_id: int, root: int, dist_out) -> int:
    """Queue a query; dist_out is a host row of int32 or int8 (then
    submitted with BFS_DIST_INT8)."""
    flags = _row_flags(dist_out)
    p, dev = _buf(dist_out)
    if dev:
        raise ValueError("dist_out must be host memory")
    t = ctypes.c_int64()
    check(_lib.lib().bfs_submit_rows(s, graph_id, int(root), p, flags, ctypes.byref(t)),
          "bfs_submit_rows")
    return t.value


def bfs_poll(s: int, ticket: int) -> int:
    return check(_lib.lib().bfs_poll(s, ticket), "bfs_poll")


def bfs_wait(s: int, ticket: int, timeout_us: int = -1) -> int:
    return check(_lib.lib().bfs_wait(s, ticket, timeout_us), "bfs_wait")


def bfs_ticket_times(s: int, ticket: int) -> tuple[int, int, int, int]:
    """(status, submit_ns, launch_ns, done_ns) on the monotonic clock."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = check(_lib.lib().bfs_ticket_times(s, ticket, ctypes.byref(a), ctypes.byref(b),
                                           ctypes.byref(c)), "bfs_ticket_times")
    return st, a.value, b.value, c.value


def bfs_release(s: int, ticket: int) -> None:
    check(_lib.lib().bfs_release(s, ticket), "bfs_release")


def bfs_server_get_stats(s: int) -> dict:
    st = ServerStats()
    check(_lib.lib().bfs_server_get_stats(s, ctypes.byref(st)), "bfs_server_get_stats")
    return {f: getattr(st, f) for f, _ in ServerStats._fields_}


def bfs_server_replay(s: int, graph_ids, roots, arrival_ns, graph_bufs, timeout_us: int = -1):
    """Replay a query trace from native threads (see include/bfs.h).
    graph_bufs: one C-contiguous host array [k_g, n_g] per graph, all int32 or
    all int8 (then the queries ask for int8 rows; pinned memory keeps the
    copies fast).  Returns (done_ns, status, slot) arrays."""
    gid = np.ascontiguousarray(graph_ids, dtype=np.int32)
    rts = np.ascontiguousarray(roots, dtype=np.int32)
    arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    nq = len(gid)
    if len(rts) != nq or len(arr) != nq:
        raise ValueError("graph_ids, roots and arrival_ns must have the same length")
    flags = {_row_flags(b) for b in graph_bufs}
    if len(flags) != 1:
        raise TypeError("replay buffers must all be int32 or all int8")
    ptrs = (ctypes.c_void_p * len(graph_bufs))()
    counts = np.zeros(len(graph_bufs), dtype=np.int32)
    for i, b in enumerate(graph_bufs):
        p, dev = _buf(b)
        if dev:
            raise ValueError("replay buffers are host memory")
        ptrs[i] = p
        counts[i] = b.shape[0]
    done = np.zeros(nq, dtype=np.int64)
    status = np.zeros(nq, dtype=np.int32)
    slot = np.zeros(nq, dtype=np.int32)
    check(_lib.lib().bfs_server_replay_rows(s, nq, gid.ctypes.data, rts.ctypes.data,
                                            arr.ctypes.data, ctypes.cast(ptrs, ctypes.c_void_p),
                                            counts.ctypes.data, flags.pop(), int(timeout_us),
                                            done.ctypes.data, status.ctypes.data,
                                            slot.ctypes.data),
          "bfs_server_replay_rows")
    return done, status, slot


def bfs_replay_single(graphs, graph_ids, roots, arrival_ns, graph_bufs, stream=None):
    """The one-at-a-time baseline of a served trace (see include/bfs.h):
    query i runs as bfs_run with a host output row once its arrival time has
    come, in arrival order, from a native thread.  graphs: graph handles;
    graph_bufs: one C-contiguous host array [k_g, n_g] per graph, all int32 or
    all int8 (int8 rows), used round robin.  Returns (done_ns, status)
    arrays."""
    gid = np.ascontiguousarray(graph_ids, dtype=np.int32)
    rts = np.ascontiguousarray(roots, dtype=np.int32)
    arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    nq = len(gid)
    if len(rts) != nq or len(arr) != nq or len(graph_bufs) != len(graphs):
        raise ValueError("graph_ids, roots and arrival_ns must have the same length, "
                         "and one buffer array per graph")
    hs = (ctypes.c_void_p * len(graphs))(*graphs)
    flags = {_row_flags(b) for b in graph_bufs}
    if len(flags) != 1:
        raise TypeError("replay buffers must all be int32 or all int8")
    ptrs = (ctypes.c_void_p * len(graph_bufs))()
    counts = np.zeros(len(graph_bufs), dtype=np.int32)
    for i, b in enumerate(graph_bufs):
        p, dev = _buf(b)
        if dev:
            raise ValueError("replay buffers are host memory")
        ptrs[i] = p
        counts[i] = b.shape[0]
    done = np.zeros(nq, dtype=np.int64)
    status = np.zeros(nq, dtype=np.int32)
    check(_lib.lib().bfs_replay_single(ctypes.cast(hs, ctypes.c_void_p), len(graphs), nq,
                                       gid.ctypes.data, rts.ctypes.data, arr.ctypes.data,
                                       ctypes.cast(ptrs, ctypes.c_void_p), counts.ctypes.data,
                                       flags.pop(), _stream(stream), done.ctypes.data,
                                       status.ctypes.data),
          "bfs_replay_single")
    return done, status


def bfs_server_destroy(s: int) -> None:
    check(_lib.lib().bfs_server_destroy(s), "bfs_server_destroy")


# ----------------------------------------------------- small conveniences

class Context:
    def __init__(self, device: int = 0, arena=None):
        self._arena = arena
        self.handle = bfs_context_create(device, arena)

    def close(self):
        if self.handle:
            bfs_context_destroy(self.handle)
            self.handle = None

    def run_paths(self, row_off, col, root: int, hops, sigma, weight=None, lo: int = 0,
                  hi: int = 0, stream=None) -> dict:
        return bfs_run_paths(self.handle, row_off, col, root, hops, sigma, weight, lo, hi, stream)

    def memory(self) -> tuple[int, int]:
        used, cap = ctypes.c_size_t(), ctypes.c_size_t()
        check(_lib.lib().bfs_context_memory(self.handle, ctypes.byref(used), ctypes.byref(cap)),
              "bfs_context_memory")
        return used.value, cap.value

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    def __init__(self, ctx: Context, row_off, col, flags: int = 0, stream=None):
        self.ctx = ctx
        self.handle = bfs_graph_upload(ctx.handle, row_off, col, flags, stream)
        self.n = (row_off.shape[0] if hasattr(row_off, "shape") else len(row_off)) - 1

    def info(self) -> dict:
        return bfs_graph_get_info(self.handle)

    def set_bins(self, t_small, t_large, chunk_warp, chunk_cta):
        bfs_graph_set_bins(self.handle, t_small, t_large, chunk_warp, chunk_cta)

    def autotune(self, roots, batched: bool = False, cache_path: str | None = None) -> dict:
        return bfs_graph_autotune(self.handle, roots, batched, cache_path)

    def set_option(self, option: int, value: int):
        bfs_graph_set_option(self.handle, option, value)

    def run(self, root, dist, parent=None, stream=None, flags=0):
        bfs_run(self.handle, root, dist, parent, stream, flags)

    def sync(self, stream=None) -> dict:
        return bfs_graph_sync(self.handle, stream)

    def run_lrb(self, root, dist, stream=None) -> dict:
        return bfs_run_lrb(self.handle, root, dist, stream)

    def run_butterfly(self, root, nodes, fanout, dist, stream=None) -> dict:
        return bfs_run_butterfly(self.handle, root, nodes, fanout, dist, stream)

    def run_batch(self, roots, dist, stream=None, flags=0):
        bfs_run_batch(self.handle, roots, dist, stream, flags)

    def batch_sync(self, stream=None) -> dict:
        return bfs_batch_sync(self.handle, stream)

    def close(self):
        if self.handle:
            bfs_graph_free(self.handle)
            self.handle = None


class Server:
    def __init__(self, ctx: Context, memory_budget: int, num_streams: int = 4):
        self.handle = bfs_server_create(ctx.handle, memory_budget, num_streams)

    def add_graph(self, g: Graph) -> int:
        return bfs_server_add_graph(self.handle, g.handle)

    def submit(self, graph_id: int, root: int, dist_out) -> int:
        return bfs_submit(self.handle, graph_id, root, dist_out)

    def poll(self, ticket: int) -> int:
        return bfs_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_us: int = -1) -> int:
        return bfs_wait(self.handle, ticket, timeout_us)

    def release(self, ticket: int) -> None:
        bfs_release(self.handle, ticket)

    def times(self, ticket: int) -> tuple[int, int, int, int]:
        return bfs_ticket_times(self.handle, ticket)

    def stats(self) -> dict:
        return bfs_server_get_stats(self.handle)

    def replay(self, graph_ids, roots, arrival_ns, graph_bufs, timeout_us: int = -1):
        return bfs_server_replay(self.handle, graph_ids, roots, arrival_ns, graph_bufs, timeout_us)

    def close(self):
        if self.handle:
            bfs_server_destroy(self.handle)
            self.handle = None
