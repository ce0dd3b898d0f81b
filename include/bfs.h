/*
 * bfs.h -- C ABI of the GB300 breadth-first-search library (libbfs.so).
 *
 * The library runs the per-GPU top-down level step of ButterFly BFS
 * (Green, "ButterFly BFS - An Efficient Communication Pattern for Multi
 * Node Traversals", arXiv 2103.13577): Algorithm 2 Phase 1 with one compute
 * node, which is Algorithm 1 with an atomic enqueue -- expand every frontier
 * vertex's adjacency list, claim each unvisited neighbour exactly once,
 * write its distance (level + 1), and build the next frontier.  On top of
 * that it offers 64-root batched traversal and a query server.
 *
 * Conventions shared by every entry point
 *   - Graphs are CSR: row_off int64[n+1] (row_off[0] = 0, non-decreasing,
 *     row_off[n] = nnz) and col int32[nnz] with 0 <= col[e] < n.  Edge
 *     (v, col[e]) for row_off[v] <= e < row_off[v+1] is directed v -> col[e]
 *     (Section "Preliminaries": an undirected graph stores both directions).
 *     Duplicates and self-loops are allowed and harmless; nothing is repaired.
 *   - Distances are int32 (int8 where a flag says so): d[root] = 0, d[v] =
 *     hops of a shortest path root -> v, and -1 for "infinity" (no path).
 *   - Parents: parent[root] = root, -1 when unreached, otherwise some vertex
 *     p with an edge p -> v and d[p] = d[v] - 1.  When several such p exist,
 *     which one is returned is unspecified.
 *   - Streams are cudaStream_t values passed as void* (NULL = legacy default
 *     stream).  A call with device outputs only enqueues work and returns;
 *     a call with any host buffer also waits for that stream.
 *   - Every call returns a bfs_status; nothing throws across the ABI.
 *     bfs_last_error() gives a message for the calling thread's last failure.
 *   - Pointers stay owned by the caller unless a function says otherwise.
 */
#ifndef BFS_H
#define BFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t bfs_status;

#define BFS_OK                  0
#define BFS_PENDING             1   /* bfs_poll: query not finished yet */
#define BFS_ERR_INVALID_ARG    -1   /* null pointer, bad size or flag */
#define BFS_ERR_INVALID_GRAPH  -2   /* CSR fails the checks listed above */
#define BFS_ERR_ROOT_RANGE     -3   /* root < 0 or root >= n */
#define BFS_ERR_NO_MEMORY      -4   /* device allocation (or arena) exhausted */
#define BFS_ERR_BUDGET         -5   /* server: query can never fit the budget */
#define BFS_ERR_DEPTH_OVERFLOW -6   /* int8 distances: a level above 126 */
#define BFS_ERR_TIMEOUT        -7   /* a bounded device-side wait gave up */
#define BFS_ERR_CUDA           -8   /* CUDA runtime error (message has it) */
#define BFS_ERR_UNSUPPORTED    -9   /* graph too large for the encoding */
#define BFS_ERR_CANCELLED     -10   /* server shut down before the query ran */
#define BFS_ERR_NOT_FOUND     -11   /* unknown ticket or graph id */

typedef struct bfs_context bfs_context;
typedef struct bfs_graph bfs_graph;
typedef struct bfs_server bfs_server;
typedef int64_t bfs_ticket;

/* ---- flags ------------------------------------------------------------ */
/* bfs_graph_upload */
#define BFS_UPLOAD_DEVICE_PTRS  0x1u  /* row_off/col are device pointers */
#define BFS_UPLOAD_NO_RELABEL   0x2u  /* keep the caller's vertex order on device */
/* bfs_run / bfs_run_batch */
#define BFS_OUT_HOST            0x1u  /* outputs are host pointers (copied back, call waits) */
#define BFS_DIST_INT8           0x2u  /* int8 distances (levels <= 126): bfs_run_batch,
                                         bfs_run, bfs_submit_rows and the replays */
#define BFS_HOST_LOOP           0x4u  /* one kernel launch per level, host reads the frontier
                                         size between levels (no device-side loop) */
#define BFS_GRAPH_LOOP          0x8u  /* the level loop as a CUDA graph: init, seed, then a
                                         conditional while node whose body (the level's
                                         kernels and a one-CTA step that sets the condition
                                         from the next frontier's size) repeats on the device;
                                         no cooperative launch, no host round trip.  The
                                         instantiated graph is kept per graph and output
                                         buffers and reused with new roots. */

/* ---- context ------------------------------------------------------------
 * A context binds the library to one CUDA device.  arena (device pointer,
 * may be NULL) and arena_bytes let the caller hand over one pre-allocated
 * device buffer (for instance a torch uint8 tensor); every device buffer the
 * library needs is then carved from it and nothing else is allocated.  With
 * arena == NULL the library calls cudaMalloc itself.  The arena stays owned
 * by the caller and must outlive the context. */
bfs_status bfs_context_create(int device, void* arena, size_t arena_bytes, bfs_context** out);
bfs_status bfs_context_destroy(bfs_context* ctx);
/* bytes of device memory the context currently holds (arena or cudaMalloc) */
bfs_status bfs_context_memory(const bfs_context* ctx, size_t* used, size_t* capacity);

/* ---- graphs ---------------------------------------------------------------
 * bfs_graph_upload copies the CSR to the device (host or device source per
 * flags), checks it (BFS_ERR_INVALID_GRAPH), and sizes every per-traversal
 * buffer once (the paper's tight memory bound: buffers are allocated in
 * advance and reused by every level, Section "Fanout & Trade-offs" and
 * contribution 4).  Unless BFS_UPLOAD_NO_RELABEL is given, vertices are
 * renumbered on the device by decreasing degree; results are always
 * returned in the caller's numbering.  The caller may free its arrays when
 * the call returns.  stream orders the copies. */
bfs_status bfs_graph_upload(bfs_context* ctx, const int64_t* row_off, const int32_t* col,
                            int64_t n, int64_t nnz, uint32_t flags, void* stream,
                            bfs_graph** out);
bfs_status bfs_graph_free(bfs_graph* g);

typedef struct bfs_graph_info {
    int64_t n;              /* vertices */
    int64_t nnz;            /* directed adjacency entries */
    int64_t max_degree;
    int32_t t_small;        /* degree bins: deg < t_small -> warp-gather bin */
    int32_t t_large;        /* deg >= t_large -> CTA bin, otherwise warp bin */
    int32_t chunk_warp;     /* edges per base chunk of the warp bin (a work item
                               takes 1-16 base chunks, more on larger levels) */
    int32_t chunk_cta;      /* edges per base chunk of the CTA bin (1-32 per item) */
    int32_t relabelled;     /* 1 when the device copy is degree-ordered */
    int32_t grid_blocks;    /* persistent grid size used by the device loop */
    size_t device_bytes;    /* device memory held by the graph and its buffers */
} bfs_graph_info;
bfs_status bfs_graph_get_info(const bfs_graph* g, bfs_graph_info* out);

/* Degree-bin thresholds and base chunk sizes (the autotuner's knobs).
 * t_small >= 1, t_large > t_small, chunk_warp a power of two in
 * [128, 2^24], chunk_cta a power of two in [1024, 2^24] (chunk starts are
 * found with shifts).  Defaults 16, 4096, 128, 1024.  Reallocates the per-traversal buffers;
 * must not be called while a traversal on g is in flight. */
bfs_status bfs_graph_set_bins(bfs_graph* g, int32_t t_small, int32_t t_large,
                              int32_t chunk_warp, int32_t chunk_cta);

/* Per-graph tuning options (bfs_graph_set_option).  A single-source
 * persistent run (bfs_run without BFS_GRAPH_LOOP or BFS_HOST_LOOP) that uses
 * none of BFS_OPT_WARP_AGGREGATE, BFS_OPT_HOT_WORDS, BFS_OPT_DIRECTION,
 * BFS_OPT_BITMAP_FRONTIER, BFS_OPT_L2_PREFETCH and BFS_OPT_TMA_STAGE (the
 * defaults) runs a build of the traversal kernel with those paths compiled
 * out, which keeps more of its state in registers (about 10 % faster at
 * scale 22); setting any of them switches to the full build.  Results are
 * the same either way.
 *   BFS_OPT_WARP_AGGREGATE   0/1: lanes of a warp that claim vertices in the
 *                            same 32-bit visited word merge their bits and
 *                            issue one atomicOr (default 0).
 *   BFS_OPT_TIMEOUT_NS       limit of every device-side grid-barrier wait,
 *                            in ns (default 2e9); expiry ends the traversal
 *                            with BFS_ERR_TIMEOUT.
 *   BFS_OPT_CTAS_PER_SM      2, 3 or 4: resident CTAs per SM of the traversal
 *                            kernels (register cap 128, 80 or 64; batched
 *                            kernels use 3 when 4 is asked; default 4).
 *   BFS_OPT_HOT_WORDS        visited-bitmap words (multiple of 4, <= 40960)
 *                            each CTA copies to shared memory at the start of
 *                            a large level; probes of vertices below 32x that
 *                            index that were visited before the level end
 *                            there.  Default 0 (off).
 *   BFS_OPT_HOT_MIN_EDGES    a level is large when its frontier holds at least
 *                            this many adjacency entries (default 2^20).
 *   BFS_OPT_DIRECTION        0: every level top-down (Algorithm 1; default).
 *                            1: direction-optimizing -- a level runs bottom-up
 *                            (every unvisited vertex looks for a neighbour in
 *                            the frontier bitmap) when the frontier's edges
 *                            times alpha exceed the unvisited vertices' edges,
 *                            and returns to top-down when the frontier holds
 *                            fewer than n / beta vertices.  2: bottom-up on
 *                            every level (for testing).  Distances are the
 *                            same in every mode.  Batched runs (persistent
 *                            and graph loops) take the same decisions with
 *                            lane sets: a bottom-up batched level ORs the
 *                            neighbours' frontier lane sets into each vertex
 *                            until every lane it lacks is found; host-loop
 *                            batched runs stay top-down.  Modes 1 and 2 need a
 *                            symmetric graph (bottom-up follows a vertex's own
 *                            adjacency); the upload tests symmetry and other
 *                            graphs refuse them with BFS_ERR_UNSUPPORTED.
 *   BFS_OPT_DO_ALPHA, BFS_OPT_DO_BETA   the two thresholds (default 15, 18).
 *   BFS_OPT_BITMAP_FRONTIER  d > 0: a top-down level whose frontier holds more
 *                            than n / d vertices reads its light bin (deg <
 *                            t_small) from the frontier bitmap in vertex order
 *                            (tiles of 1024 vertices per warp) instead of that
 *                            bin's queue; the heavier bins keep their queues.
 *                            0: never (default).
 *   BFS_OPT_L2_PREFETCH      0/1: when a warp (bin 1) or CTA (bin 2) takes its
 *                            next batch of vertices, one bulk L2 prefetch per
 *                            vertex requests that vertex's column segment
 *                            (bin 2: its first 32 KiB, the rest 32 KiB ahead
 *                            of the reads), so the segment's reads find it in
 *                            L2 instead of each waiting on HBM.  Default 0.
 *   BFS_OPT_TMA_STAGE        0/1: heavy vertices' column runs (bin 2) are
 *                            staged in shared memory: each warp streams its
 *                            256-entry blocks of a run through two 1 KB
 *                            buffers filled by TMA bulk copies
 *                            (cp.async.bulk, completion on an mbarrier), the
 *                            next block in flight while the current one is
 *                            probed.  Costs 16 KB of shared memory per CTA.
 *                            Default 0. */
#define BFS_OPT_WARP_AGGREGATE  1
#define BFS_OPT_TIMEOUT_NS      2
#define BFS_OPT_CTAS_PER_SM     3
#define BFS_OPT_HOT_WORDS       4
#define BFS_OPT_HOT_MIN_EDGES   5
#define BFS_OPT_DIRECTION       6
#define BFS_OPT_DO_ALPHA        7
#define BFS_OPT_DO_BETA         8
#define BFS_OPT_BITMAP_FRONTIER 9
#define BFS_OPT_L2_PREFETCH     10
#define BFS_OPT_TMA_STAGE       11
bfs_status bfs_graph_set_option(bfs_graph* g, int32_t option, int64_t value);

/* ---- autotuning -----------------------------------------------------------------
 * Picks t_small, t_large, the base chunk sizes and BFS_OPT_CTAS_PER_SM for g
 * by coordinate descent (one knob at a time over a short candidate list,
 * two passes), timing each candidate with CUDA events on the sample roots
 * (host array, 1..64 entries, caller numbering): single-source runs, or one
 * batched launch with BFS_TUNE_BATCHED.  The best setting is applied to g.
 * cache_path (nullable) names a JSON-lines file: a graph whose fingerprint
 * (counts plus a hash of sampled offsets and columns) and flags are found
 * there is set up without timing; otherwise the result is appended.  Must not
 * run while other traversals on g are in flight.  The paper has no
 * autotuner; its per-bin launch sizes are fixed by the bin's degree bound. */
#define BFS_TUNE_BATCHED 0x1u
typedef struct bfs_tune_result {
    int32_t t_small, t_large, chunk_warp, chunk_cta, ctas_per_sm;
    int32_t from_cache;     /* 1 when the setting came from cache_path */
    int32_t trials;         /* candidates timed */
    double best_ms;         /* time of the chosen setting over the sample (-1 if cached) */
    uint64_t fingerprint;
} bfs_tune_result;
bfs_status bfs_graph_autotune(bfs_graph* g, const int32_t* roots, int32_t nroots, uint32_t flags,
                              const char* cache_path, bfs_tune_result* out);

/* ---- single-source traversal ----------------------------------------------
 * Algorithm 1 / Algorithm 2 Phase 1 (one compute node) from `root` (caller
 * numbering).  dist: int32[n], or int8[n] with BFS_DIST_INT8 (the int32
 * distances converted on the device; a level above 126 makes the traversal
 * report BFS_ERR_DEPTH_OVERFLOW and is written as -2); parent: int32[n] or
 * NULL.  Device pointers by
 * default (stream-ordered, returns after enqueueing); with BFS_OUT_HOST they
 * are host pointers and the call waits for completion.  Concurrent calls on
 * one graph must use the same stream (the graph's traversal buffers are
 * shared).  Errors detected on the device (timeout) are reported by the
 * next call that synchronises (BFS_OUT_HOST, bfs_graph_sync). */
bfs_status bfs_run(bfs_graph* g, int32_t root, int32_t* dist, int32_t* parent, void* stream,
                   uint32_t flags);

typedef struct bfs_run_stats {
    int64_t levels;         /* number of non-empty frontiers (max dist + 1) */
    int64_t reached;        /* vertices with dist >= 0 */
    int64_t edges_scanned;  /* m_c: sum of the out-degrees of the reached vertices --
                               the entries a top-down traversal expands and the
                               TEPS numerator in every direction mode */
    int32_t status;         /* device-side status of the last traversal */
    int32_t bottom_up_levels; /* levels run bottom-up (BFS_OPT_DIRECTION) */
} bfs_run_stats;
/* Waits for `stream`, then reports the last traversal run on g. */
bfs_status bfs_graph_sync(bfs_graph* g, void* stream, bfs_run_stats* stats);

/* ---- batched traversal ------------------------------------------------------
 * k independent traversals (1 <= k <= 64) from roots[0..k) (host array,
 * caller numbering; duplicates allowed) in one persistent launch, each vertex
 * carrying a 64-bit source-lane bitset.  dist: k rows of n (row i = the
 * distances from roots[i]), int32 by default or int8 with BFS_DIST_INT8
 * (-1 = unreached; a level above 126 makes the call fail with
 * BFS_ERR_DEPTH_OVERFLOW).  Device or host pointer as for bfs_run.
 * Each row equals bfs_run(roots[i]). */
bfs_status bfs_run_batch(bfs_graph* g, const int32_t* roots, int32_t k, void* dist,
                         void* stream, uint32_t flags);
/* Waits for `stream`, then reports the last batched traversal run on g:
 * levels = deepest lane's levels, reached = sum over lanes of reached
 * vertices, edges_scanned = sum over lanes of m_c (the batch's TEPS
 * numerator). */
bfs_status bfs_batch_sync(bfs_graph* g, void* stream, bfs_run_stats* stats);

/* ---- serving ---------------------------------------------------------------
 * A server keeps graphs resident and runs single-root queries as they
 * arrive.  Queries on the same graph that are waiting together are packed
 * into one batched launch of up to 64 lanes; when only a few wait, they run
 * as that many single-source traversals instead -- while their mean
 * completion time, t_single (k + 1) / 2, is no later than one batched
 * launch's (bfs_server_add_graph times one of each on the graph, using the
 * graph's own options, e.g. BFS_OPT_DIRECTION).  Launches run on num_streams CUDA
 * streams so work from different graphs overlaps on the device.  A launch is
 * admitted only while the device memory of all launches in flight stays
 * within memory_budget bytes; it takes as many CTAs per SM as fit next to
 * the CTAs of the launches whose kernels are still running (registers,
 * threads, shared memory; the whole grid when nothing else runs), and waits
 * when not even one fits: every persistent grid is then resident at once
 * and none waits on another's SMs.  Queries that do not fit wait.  A query whose
 * smallest launch alone exceeds the budget fails with BFS_ERR_BUDGET.
 * dist_out (host, int32[n]) is written when the query completes; the pointer
 * must stay valid until then.  Give pinned memory (cudaHostAlloc or a pinned
 * torch tensor): a copy into pageable memory is synchronous, so the
 * dispatcher would wait for each launch to finish before taking the next
 * queries, and nothing would overlap. */
bfs_status bfs_server_create(bfs_context* ctx, size_t memory_budget, int32_t num_streams,
                             bfs_server** out);
bfs_status bfs_server_add_graph(bfs_server* s, bfs_graph* g, int32_t* graph_id);
bfs_status bfs_submit(bfs_server* s, int32_t graph_id, int32_t root, int32_t* dist_out,
                      bfs_ticket* ticket);
/* bfs_submit with a choice of row type: flags = BFS_DIST_INT8 makes dist_out an
 * int8[n] row (a quarter of the bytes to copy to the host; levels above 126
 * fail the query with BFS_ERR_DEPTH_OVERFLOW, and the other queries of its
 * launch with it), 0 an int32[n] row as bfs_submit.  int8 and int32 queries
 * of one graph wait in separate FIFOs and never share a launch. */
bfs_status bfs_submit_rows(bfs_server* s, int32_t graph_id, int32_t root, void* dist_out,
                           uint32_t flags, bfs_ticket* ticket);
/* BFS_PENDING while queued or running, BFS_OK once dist_out is written, or
 * the query's error.  A finished ticket can be polled until it is released. */
bfs_status bfs_poll(bfs_server* s, bfs_ticket ticket);
/* Waits up to timeout_us (< 0 = no limit) for the ticket. */
bfs_status bfs_wait(bfs_server* s, bfs_ticket ticket, int64_t timeout_us);
/* Forget a finished ticket. */
bfs_status bfs_release(bfs_server* s, bfs_ticket ticket);
/* Timestamps of a ticket on the monotonic clock (CLOCK_MONOTONIC, ns):
 * submission, launch of the batch that carried it, and completion as seen
 * by the server (0 while not reached).  Returns the ticket's status. */
bfs_status bfs_ticket_times(bfs_server* s, bfs_ticket ticket, int64_t* submit_ns,
                            int64_t* launch_ns, int64_t* done_ns);

typedef struct bfs_server_stats {
    int64_t submitted, completed, failed;
    int64_t launches;         /* batched launches issued */
    int64_t lanes;            /* queries carried by those launches */
    int64_t max_inflight_bytes;
} bfs_server_stats;
bfs_status bfs_server_get_stats(bfs_server* s, bfs_server_stats* out);

/* Replays a query trace against the server from native threads (load
 * generation with nothing of the caller's runtime in the loop).  Query i is
 * submitted at arrival_ns[i] (steady clock, the clock of bfs_ticket_times;
 * non-decreasing) on graph graph_ids[i] with root roots[i].  Its row goes to
 * one of bufs_per_graph[g] host buffers of graph g: graph_bufs[g] points to
 * bufs_per_graph[g] consecutive rows of n_g int32 (pinned memory keeps the
 * copies fast); a query takes any free buffer of its graph and waits for
 * one to come back if none is free (a buffer returns when its query
 * completes).  On return (every query done) done_ns[i] is the query's
 * completion time on the server's clock, status_out[i] its status and, when
 * slot_out is not NULL, slot_out[i] the buffer it used.  Each graph's
 * queries are submitted by a thread of their own, so a graph whose buffers
 * are all in use delays only its own later queries.  Waits inside are
 * bounded by timeout_us per query (negative: none). */
bfs_status bfs_server_replay(bfs_server* s, int64_t nq, const int32_t* graph_ids,
                             const int32_t* roots, const int64_t* arrival_ns,
                             int32_t* const* graph_bufs, const int32_t* bufs_per_graph,
                             int64_t timeout_us, int64_t* done_ns, int32_t* status_out,
                             int32_t* slot_out);
/* bfs_server_replay with int8 rows when flags = BFS_DIST_INT8 (graph_bufs[g]
 * then holds bufs_per_graph[g] rows of n_g int8; every query is submitted
 * with bfs_submit_rows and those flags). */
bfs_status bfs_server_replay_rows(bfs_server* s, int64_t nq, const int32_t* graph_ids,
                                  const int32_t* roots, const int64_t* arrival_ns,
                                  void* const* graph_bufs, const int32_t* bufs_per_graph,
                                  uint32_t flags, int64_t timeout_us, int64_t* done_ns,
                                  int32_t* status_out, int32_t* slot_out);
/* The one-at-a-time baseline of a served trace: query i (graph
 * graphs[graph_ids[i]], root roots[i]) runs as bfs_run with a host output
 * row (BFS_OUT_HOST on `stream`) once arrival_ns[i] has come, strictly in
 * arrival order, from the calling thread -- each query waits for every
 * earlier one, as repeated plain single-source traversals on one GPU do.
 * Rows go to graph_bufs[g] (bufs_per_graph[g] consecutive rows of n_g int32,
 * or int8 with flags = BFS_DIST_INT8, used round robin).  done_ns[i] is the
 * time bfs_run returned (steady clock, as bfs_ticket_times), status_out[i]
 * its status.  Returns the first failure, if any. */
bfs_status bfs_replay_single(bfs_graph* const* graphs, int32_t ngraphs, int64_t nq,
                             const int32_t* graph_ids, const int32_t* roots,
                             const int64_t* arrival_ns, void* const* graph_bufs,
                             const int32_t* bufs_per_graph, uint32_t flags, void* stream,
                             int64_t* done_ns, int32_t* status_out);
/* Stops the server; queued queries finish with BFS_ERR_CANCELLED. */
bfs_status bfs_server_destroy(bfs_server* s);

/* ---- ButterFly BFS emulated on one GPU -----------------------------------------
 * Algorithm 2 with `nodes` virtual compute nodes on this device: each node
 * keeps its own distance array, owns one 1D vertex range of about nnz/nodes
 * adjacency entries (Section "Graph Partitioning"), expands only its owned
 * frontier (Phase 1, atomic claim per node), then log_r(nodes) butterfly
 * rounds (Phase 2, r = max(2, fanout)): in round i a node receives the
 * global queue of every node whose base-r id differs only in digit i,
 * filters it by its own distances and enqueues the new vertices.  nodes
 * must be a power of r (1..256), fanout 1..16.  dist: device int32[n] in the
 * caller's numbering (node 0's view; every node's view is compared and the
 * differences counted).  Waits for `stream`.  Nodes run one after another:
 * this is for correctness and the message accounting of Section "Fanout &
 * Trade-offs" (messages per level = nodes * (r - 1) * rounds; a node's
 * receive buffer holds at most (r - 1) global queues, O(f * V)), not speed. */
typedef struct bfs_butterfly_stats {
    int64_t levels;
    int64_t rounds_per_level;
    int64_t messages;                  /* queue transfers between nodes */
    int64_t message_entries;           /* vertex ids carried by them */
    int64_t max_round_buffer_entries;  /* largest receive buffer of one node in one round */
    int64_t max_global_queue;          /* largest Q_global at the start of a round */
    int64_t node_disagreements;        /* (node, vertex) distances differing from node 0 */
    int32_t nodes, radix;
} bfs_butterfly_stats;
bfs_status bfs_run_butterfly(bfs_graph* g, int32_t root, int32_t nodes, int32_t fanout,
                             int32_t* dist, void* stream, bfs_butterfly_stats* stats);
/* The exchange schedule itself (host only, no device work): the nodes whose
 * global queues `node` receives in round `round` (ButterflyDirection of
 * Algorithm 2 generalised to fanout f: the ids differing from `node` only in
 * base-max(2,f) digit `round`).  partners: room for 15 ids; *count set. */
bfs_status bfs_butterfly_schedule(int32_t nodes, int32_t fanout, int32_t round, int32_t node,
                                  int32_t* partners, int32_t* count);

/* ---- the paper's load-balancing scheme, for comparison ---------------------------
 * Single-source traversal run the way Section "Load Balanced Traversals Per
 * compute-node" describes: each level the frontier is grouped by Logarithmic
 * Radix Binning (bin b: degrees in [2^(b-1), 2^b)), one kernel per non-empty
 * bin is launched on its own stream with a thread-block shape taken from the
 * bin's degree bound (thread, warp or block per vertex), the host joins the
 * streams and reads the next frontier size.  Visited test: d[u] = infinity
 * claimed by compare-and-swap.  dist: device int32[n], caller numbering.
 * Waits for `stream`.  An ablation against bfs_run's fused persistent
 * design, not a faster path. */
typedef struct bfs_lrb_stats {
    int64_t levels;
    int64_t kernels;   /* bin kernels launched */
} bfs_lrb_stats;
bfs_status bfs_run_lrb(bfs_graph* g, int32_t root, int32_t* dist, void* stream,
                       bfs_lrb_stats* stats);

/* ---- shortest-path counts and weight-filtered traversal -------------------------
 * Section "Top Down Vs. Bottom Up" names two uses of BFS that need every
 * entry leaving the frontier examined (so no bottom-up level): counting all
 * shortest paths, as betweenness centrality does, and weight-filtering BFS,
 * which follows only edges of given weights.  This call does both, top-down:
 * on the subgraph of the CSR entries e with w_lo <= weight[e] <= w_hi (every
 * entry when weight is NULL; w_lo > w_hi keeps none),
 *   hops[v]  = length of a shortest root -> v path, -1 when none (int32[n]);
 *   sigma[v] = number of shortest root -> v paths (double[n]; a path is a
 *              sequence of entries, so a duplicated entry gives two paths;
 *              sigma[root] = 1, 0 where unreached) -- the forward phase of
 *              Brandes' betweenness algorithm.
 * Counts are summed with double-precision atomic adds in no fixed order:
 * exact while they stay below 2^53, otherwise within the rounding of the
 * additions (relative error below about levels x max in-degree x 2^-53).
 *
 * row_off (int64[n+1]), col (int32[nnz]; may be NULL when nnz = 0), weight
 * (int32[nnz] or NULL), hops and sigma are device pointers of ctx's GPU, in
 * the caller's own numbering and entry order; anything else (host memory,
 * another GPU) fails with BFS_ERR_INVALID_ARG before any device work.  The
 * CSR is not modified and need not be uploaded; every row is checked
 * against [0, nnz] and every kept column index against [0, n) before use,
 * and a bad one ends the call with BFS_ERR_INVALID_GRAPH (outputs then
 * undefined), never with an out-of-range access.  nnz must be below
 * 2^34 (BFS_ERR_UNSUPPORTED otherwise).  Scratch (about 40.3 bytes per
 * vertex) comes from ctx's allocator -- its arena when it has one -- and is
 * returned before the call returns.  The whole level loop runs in one
 * cooperative launch on `stream` (grid barriers between its phases, each
 * wait bounded; BFS_ERR_TIMEOUT when one gives up); the call then waits for
 * the stream and returns when the traversal is complete.  stats (nullable,
 * host): levels, reached vertices, and the entries of the reached vertices'
 * rows, kept or not (edges_scanned). */
typedef struct bfs_paths_stats {
    int64_t levels;         /* non-empty frontiers (max hops + 1) */
    int64_t reached;        /* vertices with hops >= 0 */
    int64_t edges_scanned;  /* entries of the reached vertices' rows */
} bfs_paths_stats;
bfs_status bfs_run_paths(bfs_context* ctx, const int64_t* row_off, const int32_t* col,
                         const int32_t* weight, int64_t n, int64_t nnz, int32_t w_lo,
                         int32_t w_hi, int32_t root, int32_t* hops, double* sigma, void* stream,
                         bfs_paths_stats* stats);

/* ---- traversal without device allocation ---------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory at traversal time -- code that runs inside a
 * fixed device-memory plan owned by someone else (a framework's allocator,
 * an embedded or real-time service with its memory reserved up front), or
 * that must not trigger the device-wide synchronisation cudaMalloc and
 * cudaFree can imply.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Same traversal as bfs_run, on a CSR the caller already holds on the
 * device: row_off (int64[n+1], 8-byte aligned), col (int32[nnz], 16-byte
 * aligned; whole 16-byte blocks are read, so the tail of the block holding
 * the last entry must be readable, as it is for any cudaMalloc or torch
 * buffer), dist (int32[n]) and parent (int32[n] or NULL) are device pointers
 * on the calling thread's current device; stream as for bfs_run.  Each call
 * checks the CSR on the device before the traversal reads it (one extra pass
 * over row_off and col): offsets must not decrease, row_off[0] >= 0,
 * row_off[n] <= nnz, and every col[e] (0 <= e < nnz) must lie in [0, n).  A
 * CSR that fails the check ends the traversal before any index is used and
 * the call reports BFS_ERR_INVALID_GRAPH (dist and parent are then left as
 * they were).
 *
 * Scratch: one fixed array of about 30 MB in the library's device code,
 * reserved on every GPU that loads the library and held until the process
 * exits; graphs are limited to n <= 524,288 vertices and nnz <= 33,554,432
 * entries, larger ones fail with BFS_ERR_UNSUPPORTED.  The first successful
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and the kernel's occupancy and keeps them for the process; make that first
 * call before any stream capture (a failed set-up is not kept and is tried
 * again by the next call), and do not call the function on a device after
 * cudaDeviceReset there (the kept address would be stale).  All calls share
 * the one array and each call clears what must start at zero, so calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads, without ordering between them) race and give undefined results:
 * order them on one stream.  With stats == NULL the call only enqueues the
 * work and device-side failures (a failed CSR check, an expired wait) are
 * not reported to the caller; pass a host stats pointer to have the call
 * wait for the stream, report the traversal, and return BFS_ERR_INVALID_GRAPH
 * or BFS_ERR_TIMEOUT when the device recorded one. */
bfs_status bfs_run_static(const int64_t* row_off, const int32_t* col, int64_t n, int64_t nnz,
                          int32_t root, int32_t* dist, int32_t* parent, void* stream,
                          bfs_run_stats* stats);

/* ---- diagnostics ------------------------------------------------------------ */
const char* bfs_last_error(void);
const char* bfs_status_string(bfs_status s);
int32_t bfs_version(void);

/* Fault-detection hook for tests: makes the next device-side grid barrier
 * on g wait for an arrival that never comes, so the bounded wait (limit
 * timeout_ns) expires and the traversal ends with BFS_ERR_TIMEOUT.  The
 * kernel returns normally; the context stays usable.  timeout_ns = 0
 * restores normal operation (default limit). */
bfs_status bfs_debug_set_barrier_test(bfs_graph* g, int32_t stall, int64_t timeout_ns);

/* Level timeline of the persistent traversals (bfs_run and bfs_run_batch
 * without BFS_HOST_LOOP).  d_stamps: device array of cap >= 3 uint64
 * entries, owned by the caller and kept alive while traversals run; nullptr
 * turns the timeline off (default).  Each traversal writes %globaltimer (ns)
 * into d_stamps[0] at kernel start, [1] after the initialisation barrier,
 * [2] after the roots are seeded, then single-source: [3 + L] after level
 * L's barrier; batched: [3 + 2L] after level L's expansion and [4 + 2L]
 * after its sweep -- for as many entries as fit; later entries are left
 * unwritten.  The timestamps cost one store per barrier. */
bfs_status bfs_debug_set_timeline(bfs_graph* g, uint64_t* d_stamps, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* BFS_H */
