// bfs_runtime.h -- host-side runtime objects behind the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>

#include "../../include/bfs.h"
#include "bfs_internal.h"

namespace bfs {

// Device-memory source of a context: the caller's arena (first-fit free
// list, 256-byte granules, coalescing on free) or cudaMalloc.
class DeviceAllocator {
public:
    DeviceAllocator(void* arena, size_t bytes);
    ~DeviceAllocator();
    void* alloc(size_t bytes);           // nullptr when exhausted
    void release(void* p);
    size_t used() const;
    size_t capacity() const;

private:
    mutable std::mutex mu_;
    char* base_;
    size_t cap_;
    size_t used_ = 0;
    std::map<size_t, size_t> free_;      // offset -> size (arena mode)
    std::map<void*, size_t> live_;       // pointer -> size
};

// Per-traversal buffers of one graph: everything one launch touches besides
// the graph itself and the caller's outputs.  Sized once from the degree
// histogram (the paper's tight bound: no allocation inside the level loop).
struct Workspace {
    bool batched = false;
    size_t bytes = 0;
    uint32_t* visited = nullptr;
    BinQueue q[2][kBins];
    char* control = nullptr;           // LevelCtl[3] | GridBarrier | DevStats
    LevelCtl* ctl = nullptr;
    GridBarrier* bar = nullptr;
    DevStats* stats = nullptr;
    uint32_t* fb[3] = {nullptr, nullptr, nullptr};  // plain: frontier bitmaps
    uint64_t* lane_vn = nullptr;       // batched: [n][2] visited / next lane sets
    uint64_t* lane_front = nullptr;    // batched: [n] frontier lane sets (bottom-up levels)
    uint8_t* lane_level = nullptr;     // batched: [n][64] level bytes
    int32_t* roots = nullptr;          // [64]
    int32_t* dist_scratch = nullptr;   // host-output staging (plain: n; batched: none)
    int8_t* dist8_scratch = nullptr;   // plain int8 rows with host output: n bytes
    int32_t* parent_scratch = nullptr;
    void* batch_dist_scratch = nullptr;  // batched host-output staging, 64 * n int32
    DeviceAllocator* mem = nullptr;    // where the buffers came from
};

}  // namespace bfs

struct bfs_context {
    int device = 0;
    int sms = 0;
    size_t l2_bytes = 0;
    bfs::DeviceAllocator* mem = nullptr;
};

namespace bfs {
struct GraphLoop;  // an instantiated graph-captured level loop (BFS_GRAPH_LOOP)
}

struct bfs_graph {
    bfs::GraphLoop* loop_plain = nullptr;
    bfs::GraphLoop* loop_batch = nullptr;
    bfs_context* ctx = nullptr;
    int64_t n = 0, nnz = 0, max_degree = 0;
    int64_t* d_off = nullptr;
    int32_t* d_col = nullptr;
    int32_t* d_new2old = nullptr;     // device numbering -> caller numbering
    int32_t* d_old2new = nullptr;     // caller numbering -> device numbering
    bool relabelled = false;
    int32_t t_small = 16, t_large = 4096, chunk_warp = 128, chunk_cta = 1024;
    uint64_t bin_count[bfs::kBins] = {0, 0, 0};
    uint64_t bin_edges[bfs::kBins] = {0, 0, 0};
    bfs::Workspace* ws_plain = nullptr;
    bfs::Workspace* ws_batch = nullptr;
    size_t graph_bytes = 0;
    int32_t grid_plain = 0, grid_batch = 0;
    int32_t debug_stall = 0;
    long long timeout_ns = 2000000000ll;
    int32_t use_match_any = 0;
    int32_t min_blocks = 4;           // resident CTAs per SM the kernels are built for
    int32_t hot_words = 0;            // visited words kept in shared memory on large levels
    long long hot_min_edges = 1ll << 20;
    int32_t dir_mode = 0;             // 0 top-down, 1 direction-optimizing, 2 bottom-up always
    int32_t do_alpha = 15, do_beta = 18;
    int32_t bitmap_div = 0;           // bitmap top-down when frontier > n / bitmap_div
    int32_t l2_prefetch = 0;          // bulk L2 prefetch of bin 1 / bin 2 column segments
    int32_t tma_stage = 0;            // bin-2 blocks staged in shared memory by TMA
    uint64_t* timeline = nullptr;     // diagnostics: device array of level timestamps
    int32_t timeline_cap = 0;
    int64_t n_nonzero = 0;            // vertices with out-degree > 0
    bool symmetric = false;           // every edge stored in both directions
    std::mutex mu;
};

namespace bfs {
// NVTX range in the library's own domain ("bfs"), with an integer payload
// (root, lane count, level ...): the host side of every traversal, upload,
// tuning trial, host-driven level and server launch shows up by name on an
// Nsight timeline.  With no tool attached a push/pop is a pointer test.
class TraceRange {
public:
    TraceRange(const char* name, int64_t payload = 0) {
        static nvtxDomainHandle_t dom = nvtxDomainCreateA("bfs");
        domain_ = dom;
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
        a.payload.llValue = payload;
        nvtxDomainRangePushEx(domain_, &a);
    }
    ~TraceRange() { nvtxDomainRangePop(domain_); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;

private:
    nvtxDomainHandle_t domain_;
};

// helpers shared by the C ABI translation units
void set_error(const std::string& msg);
bfs_status cuda_fail(cudaError_t e, const char* what);
Workspace* make_workspace(bfs_graph* g, DeviceAllocator* m, bool batched, cudaStream_t s,
                          bfs_status* st);
void free_workspace(bfs_graph* g, Workspace* ws);
size_t workspace_bytes(const bfs_graph* g, bool batched, int nlanes);
bfs_status run_batch_on(bfs_graph* g, Workspace* ws, const int32_t* roots, int32_t k, void* dist,
                        cudaStream_t stream, uint32_t flags, int32_t grid);
bfs_status batch_finish(bfs_graph* g, Workspace* ws, cudaStream_t stream, bfs_run_stats* stats);
bfs_status run_plain_on(bfs_graph* g, Workspace* ws, int32_t root, int32_t* dist, int32_t* parent,
                        cudaStream_t stream, uint32_t flags, int32_t grid);
int32_t plain_grid_of(const bfs_graph* g);
// Resources one CTA of g's persistent traversal kernel holds on an SM
// (registers, threads, shared memory), for launches that share the GPU.
struct CtaFootprint {
    int regs = 0;
    int threads = 0;
    size_t smem = 0;
};
bfs_status cta_footprint(const bfs_graph* g, bool batched, CtaFootprint* out);
// int8 copy of k rows of n int32 distances (-1 stays -1); a distance above
// 126 records kDevDepth in stats (when not null) and is written as -2
cudaError_t launch_dist_to_int8(const int32_t* src, int8_t* dst, long long count, DevStats* stats,
                                int sms, cudaStream_t s);
}  // namespace bfs
