"""GB300-native breadth-first search (ButterFly BFS per-GPU level step).

Thin Python binding over the C ABI of ``libbfs.so`` (``include/bfs.h``):
the functions below carry the C names and only marshal arguments (numpy
arrays -> host pointers, torch CUDA tensors -> device pointers, torch
streams -> cudaStream_t).  Every step of a traversal runs in the library's
CUDA kernels; there is no CPU fallback -- loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    BFS_DIST_INT8,
    BFS_ERR_BUDGET,
    BFS_ERR_CANCELLED,
    BFS_ERR_CUDA,
    BFS_ERR_DEPTH_OVERFLOW,
    BFS_ERR_INVALID_ARG,
    BFS_ERR_INVALID_GRAPH,
    BFS_ERR_NO_MEMORY,
    BFS_ERR_NOT_FOUND,
    BFS_ERR_ROOT_RANGE,
    BFS_ERR_TIMEOUT,
    BFS_ERR_UNSUPPORTED,
    BFS_GRAPH_LOOP,
    BFS_HOST_LOOP,
    BFS_OPT_BITMAP_FRONTIER,
    BFS_OPT_CTAS_PER_SM,
    BFS_OPT_DIRECTION,
    BFS_OPT_DO_ALPHA,
    BFS_OPT_DO_BETA,
    BFS_OPT_HOT_MIN_EDGES,
    BFS_OPT_HOT_WORDS,
    BFS_OPT_L2_PREFETCH,
    BFS_OPT_TMA_STAGE,
    BFS_OPT_TIMEOUT_NS,
    BFS_OPT_WARP_AGGREGATE,
    BFS_OK,
    BFS_OUT_HOST,
    BFS_PENDING,
    BFS_TUNE_BATCHED,
    BFS_UPLOAD_DEVICE_PTRS,
    BFS_UPLOAD_NO_RELABEL,
    BfsError,
    lib,
    load,
)
from .api import (  # noqa: F401
    Context,
    Graph,
    Server,
    bfs_batch_sync,
    bfs_butterfly_schedule,
    bfs_context_create,
    bfs_context_destroy,
    bfs_debug_set_timeline,
    bfs_graph_autotune,
    bfs_graph_free,
    bfs_graph_get_info,
    bfs_graph_set_bins,
    bfs_graph_set_option,
    bfs_graph_sync,
    bfs_graph_upload,
    bfs_poll,
    bfs_release,
    bfs_run,
    bfs_run_batch,
    bfs_run_butterfly,
    bfs_run_lrb,
    bfs_run_static,
    bfs_server_add_graph,
    bfs_server_create,
    bfs_server_destroy,
    bfs_server_get_stats,
    bfs_server_replay,
    bfs_submit,
    bfs_ticket_times,
    bfs_wait,
)
