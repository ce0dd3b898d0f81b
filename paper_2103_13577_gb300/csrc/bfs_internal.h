// bfs_internal.h -- structures shared by the kernels and the host runtime.
#pragma once

#include <cstddef>
#include <cstdint>

namespace bfs {

constexpr int kBlock = 256;               // threads per CTA of every traversal kernel
constexpr int kWarps = kBlock / 32;
constexpr int kBins = 3;                  // 0: warp-gather, 1: warp-per-vertex, 2: CTA chunks
constexpr int kCountShift = 34;           // packed bin counter: (count << 34) | edges
constexpr unsigned long long kEdgeMask = (1ull << kCountShift) - 1ull;
constexpr int64_t kMaxVertices = (1ll << 30) - 1;    // count field holds 30 bits
constexpr int64_t kMaxEdges = (1ll << kCountShift) - 1;

// Device status codes (mirrors of BFS_ERR_* that the kernels can raise).
enum DevStatus : int { kDevOk = 0, kDevTimeout = 1, kDevOverflow = 2, kDevDepth = 3,
                       kDevInvalidGraph = 4 };

// One slot of the per-level control block; three slots rotate by level so
// that the slot being written (next frontier), the slot being read (current
// frontier) and the slot being cleared never coincide.
struct LevelCtl {
    unsigned long long packed[kBins];  // per bin: (entries << 34) | sum of degrees
    unsigned int work;                  // dynamic work-item counter of this level
    unsigned int discovered;            // vertices claimed at this level (any degree)
    unsigned long long new_lanes;       // batched: (vertex, lane) pairs discovered
    unsigned long long front_lanes;     // batched: lanes with a non-empty frontier
    unsigned long long pad[1];
};

struct GridBarrier {
    unsigned long long arrived;   // arrivals since the launch began; bit 63: a CTA gave up
    unsigned int exited;          // CTAs that have left the launch
    unsigned int pad[29];
};

struct DevStats {
    long long levels;
    long long reached;
    long long edges;
    int status;       // sticky result of the launch (read by the host)
    int max_level;
    int abort;        // set with status; tells waiting CTAs to leave; cleared at kernel exit
    int bu_levels;    // levels run bottom-up
    int pad[2];
    // graph-captured level loop: the state the device-side loop keeps in
    // registers, carried between the loop body's launches
    long long graph_seen;  // edges of all frontiers so far
    int graph_level;       // level the next body launch expands
    int graph_prev_bu;     // the previous level ran bottom-up
    int graph_dir;         // direction of the level just expanded
    int graph_pad;
    long long full_edges;  // batched: degree sum of the vertices every lane has reached
};

// Frontier queue of one bin (one of two ping-pong copies).
struct BinQueue {
    int32_t* v;            // vertex (device numbering)
    int64_t* eoff;         // exclusive prefix of degrees inside the bin (bins 1, 2)
    int32_t* chunk;        // first entry of each edge chunk (bins 1, 2)
    uint64_t* mask;        // batched traversal: source-lane bitset of the entry
    int64_t cap;           // entries
    int64_t chunk_cap;     // chunk-start slots
};

struct TraversalParams {
    // graph (device numbering)
    int64_t n;
    const int64_t* off;
    const int32_t* col;
    const int32_t* new2old;   // device -> caller numbering (nullptr: identity)
    const int32_t* old2new;   // caller -> device numbering (nullptr: identity)
    // degree bins
    int32_t t_small;
    int32_t t_large;
    int32_t chunk_warp;
    int32_t chunk_cta;
    // workspace
    uint32_t* visited;        // plain: 1 bit per vertex
    BinQueue q[2][kBins];
    LevelCtl* ctl;            // [3]
    GridBarrier* bar;
    DevStats* stats;
    // batched traversal state
    uint64_t* lane_vn;        // [n][2]: lanes that reached v (visited), lanes reaching v next
    uint64_t* lane_front;     // [n]: lanes for which v is in the current frontier
    uint8_t* lane_level;      // [n][64]: level of each lane at each vertex
    int32_t nlanes;
    int32_t dist_int8;
    int32_t roots[64];        // caller numbering, [nlanes]
    // outputs (caller numbering)
    int32_t* dist;            // plain: [n]; batched: [nlanes][n] (int32 or int8)
    int32_t* parent;          // plain only, nullable
    int32_t root_caller;      // plain: caller numbering
    // control
    int32_t level;            // host-loop mode: the level this launch runs
    int32_t phase;            // host-loop mode: 0 init, 1 seed, 2 level (batched: 3 sweep)
    long long timeout_ns;
    int32_t debug_stall;
    int32_t use_match_any;    // warp-aggregated atomicOr on the visited bitmap
    int32_t hot_words;        // visited words copied to shared memory on large levels (0: off)
    long long hot_min_edges;  // a level is large when its frontier has this many edges
    // frontier bitmaps and the bottom-up step (plain traversal)
    uint32_t* fb[3];          // frontier of level L in fb[L % 3]; nullptr: not kept
    long long nnz;
    long long bu_limit;       // bottom-up scans vertices [0, bu_limit)
    int32_t dir_mode;         // 0 top-down, 1 direction-optimizing, 2 bottom-up on every level
    int32_t do_alpha;         // top-down -> bottom-up when frontier edges * alpha > unvisited edges
    int32_t do_beta;          // bottom-up -> top-down when frontier vertices * beta < n
    int32_t dir_override;     // host-loop launches: direction chosen by the host (-1: device)
    int32_t bitmap_div;       // top-down levels with more than n / bitmap_div frontier
                              // vertices walk the frontier bitmap (0: never)
    long long bitmap_from;    // first vertex that can be light (degree-ordered graphs)
    int32_t l2_prefetch;      // bulk L2 prefetch of the heavy bins' column segments
    int32_t tma_stage;        // bin-2 column blocks staged in shared memory by TMA bulk copies
    int32_t tma_offset;       // byte offset of the staging buffers in dynamic shared memory
    int32_t timeline_cap;     // entries of timeline
    unsigned long long* timeline;  // nullable: %globaltimer after init, seed and each level
    unsigned long long graph_cond; // graph-captured loop: conditional handle of the while node
    const int* pre_status;    // nullable: a status written by an earlier launch on the same
                              // stream (CSR validation); non-zero ends the traversal before
                              // its first access to the graph
};

// Direction of level L (Beamer, Asanovic, Patterson, "Direction-optimizing
// breadth-first search", SC 2012): 0 = top-down over the frontier queues,
// 1 = top-down over the frontier bitmap, 2 = bottom-up.  m_f: edges of the
// frontier, m_u: edges of the vertices not yet visited, n_f: frontier
// vertices.
__host__ __device__ inline int choose_direction(int mode, bool prev_bu, long long m_f,
                                                long long m_u, long long n_f, long long n,
                                                int alpha, int beta, int bitmap_div) {
    const int td = (bitmap_div > 0 && n_f * (long long)bitmap_div > n) ? 1 : 0;
    if (mode == 0) return td;
    if (mode == 2) return 2;
    if (!prev_bu) return (m_f * (long long)alpha > m_u) ? 2 : td;
    return (n_f * (long long)beta < n) ? td : 2;
}

}  // namespace bfs
