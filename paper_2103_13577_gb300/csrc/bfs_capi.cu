// bfs_capi.cu -- the C ABI (include/bfs.h): contexts, device memory, graph
// upload, workspaces and the launchers of the traversal kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bfs_runtime.h"

namespace bfs {

// kernels and launch helpers (bfs_kernels.cu)
const void* plain_persistent_fn(int mb, bool staged = false);
namespace lean {
const void* plain_persistent_fn(int mb);
}
const void* plain_step_fn(int mb, bool staged = false);
const void* batch_persistent_fn(int mb);
const void* batch_step_fn(int mb);
cudaError_t launch_csr_check(const int64_t* off, const int32_t* col, long long n, long long nnz,
                             int* flags, int sms, cudaStream_t s);
cudaError_t launch_symmetry_hash(const int64_t* off, const int32_t* col, long long n,
                                 unsigned long long* sums, int sms, cudaStream_t s);
cudaError_t launch_degree_bins(const int64_t* off, long long n, int t_small, int t_large,
                               unsigned long long* counts, unsigned long long* edges,
                               unsigned long long* maxdeg, int sms, cudaStream_t s);

size_t relabel_scratch_bytes(long long n);
cudaError_t relabel_graph(const int64_t* off, const int32_t* col, long long n, long long nnz,
                          int sms, int32_t* new2old, int32_t* old2new, int64_t* new_off,
                          int32_t* new_col, void* scratch, cudaStream_t s);

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

bfs_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return BFS_ERR_CUDA;
}

static bfs_status fail(bfs_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

// ------------------------------------------------------------ allocator
static constexpr size_t kAlign = 256;
static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

DeviceAllocator::DeviceAllocator(void* arena, size_t bytes)
    : base_(static_cast<char*>(arena)), cap_(arena ? bytes : 0) {
    if (base_) {
        const size_t lead = round_up(reinterpret_cast<uintptr_t>(base_), kAlign) -
                            reinterpret_cast<uintptr_t>(base_);
        if (lead < cap_) free_[lead] = (cap_ - lead) / kAlign * kAlign;
    }
}

DeviceAllocator::~DeviceAllocator() {
    if (!base_)
        for (auto& kv : live_) cudaFree(kv.first);
}

void* DeviceAllocator::alloc(size_t bytes) {
    std::lock_guard<std::mutex> lk(mu_);
    const size_t need = round_up(std::max<size_t>(bytes, 1), kAlign);
    if (!base_) {
        void* p = nullptr;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        live_[p] = need;
        used_ += need;
        return p;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second >= need) {
            const size_t off = it->first, rest = it->second - need;
            free_.erase(it);
            if (rest) free_[off + need] = rest;
            void* p = base_ + off;
            live_[p] = need;
            used_ += need;
            return p;
        }
    }
    return nullptr;
}

void DeviceAllocator::release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    auto it = live_.find(p);
    if (it == live_.end()) return;
    const size_t sz = it->second;
    live_.erase(it);
    used_ -= sz;
    if (!base_) {
        cudaFree(p);
        return;
    }
    size_t off = static_cast<char*>(p) - base_, len = sz;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + len == nx->first) {
        len += nx->second;
        nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            pv->second += len;
            return;
        }
    }
    free_[off] = len;
}

size_t DeviceAllocator::used() const {
    std::lock_guard<std::mutex> lk(mu_);
    return used_;
}
size_t DeviceAllocator::capacity() const { return base_ ? cap_ : 0; }

// ------------------------------------------------------------ workspaces
static size_t control_bytes() {
    return round_up(3 * sizeof(LevelCtl), 128) + round_up(sizeof(GridBarrier), 128) +
           round_up(sizeof(DevStats), 128);
}

size_t workspace_bytes(const bfs_graph* g, bool batched, int /*nlanes*/) {
    size_t b = control_bytes();
    if (!batched) b += 4 * round_up(((g->n + 31) / 32 + 8) * 4, kAlign);  // visited + 3 frontier maps
    for (int bin = 0; bin < kBins; ++bin) {
        const size_t cap = g->bin_count[bin] + 1;
        const int64_t C = bin == 1 ? g->chunk_warp : g->chunk_cta;
        const size_t ccap = bin == 0 ? 0 : (g->bin_edges[bin] + C - 1) / C + 2;
        size_t per = round_up(cap * 4, kAlign);
        if (bin > 0) per += round_up(cap * 8, kAlign) + round_up(ccap * 4, kAlign);
        if (batched) per += round_up(cap * 8, kAlign);
        b += 2 * per;
    }
    if (batched)
        b += round_up((size_t)g->n * 16, kAlign) + round_up((size_t)g->n * 8, kAlign) +
             round_up((size_t)g->n * 64, kAlign);
    return b;
}

void free_workspace(bfs_graph* g, Workspace* ws) {
    (void)g;
    if (!ws) return;
    DeviceAllocator* m = ws->mem;
    if (!m) {
        delete ws;
        return;
    }
    m->release(ws->visited);
    for (int f = 0; f < 3; ++f) m->release(ws->fb[f]);
    for (int p = 0; p < 2; ++p)
        for (int b = 0; b < kBins; ++b) {
            m->release(ws->q[p][b].v);
            m->release(ws->q[p][b].eoff);
            m->release(ws->q[p][b].chunk);
            m->release(ws->q[p][b].mask);
        }
    m->release(ws->control);
    m->release(ws->lane_vn);
    m->release(ws->lane_front);
    m->release(ws->lane_level);
    m->release(ws->dist_scratch);
    m->release(ws->dist8_scratch);
    m->release(ws->parent_scratch);
    m->release(ws->batch_dist_scratch);
    delete ws;
}

Workspace* make_workspace(bfs_graph* g, DeviceAllocator* m, bool batched, cudaStream_t s,
                          bfs_status* st) {
    Workspace* ws = new (std::nothrow) Workspace();
    if (!ws) {
        *st = fail(BFS_ERR_NO_MEMORY, "host allocation failed");
        return nullptr;
    }
    ws->batched = batched;
    ws->mem = m;
    bool ok = true;
    auto get = [&](size_t bytes) -> void* {
        void* p = m->alloc(bytes);
        if (!p) ok = false;
        ws->bytes += round_up(std::max<size_t>(bytes, 1), kAlign);
        return p;
    };
    if (!batched) {
        ws->visited = static_cast<uint32_t*>(get(((g->n + 31) / 32 + 8) * 4));
        for (int f = 0; f < 3; ++f) ws->fb[f] = static_cast<uint32_t*>(get(((g->n + 31) / 32 + 8) * 4));
    }
    for (int p = 0; p < 2; ++p)
        for (int b = 0; b < kBins; ++b) {
            BinQueue& Q = ws->q[p][b];
            Q.cap = (int64_t)g->bin_count[b] + 1;
            const int64_t C = b == 1 ? g->chunk_warp : g->chunk_cta;
            Q.chunk_cap = b == 0 ? 0 : ((int64_t)g->bin_edges[b] + C - 1) / C + 2;
            Q.v = static_cast<int32_t*>(get(Q.cap * 4));
            if (b > 0) {
                Q.eoff = static_cast<int64_t*>(get(Q.cap * 8));
                Q.chunk = static_cast<int32_t*>(get(Q.chunk_cap * 4));
            }
            if (batched) Q.mask = static_cast<uint64_t*>(get(Q.cap * 8));
        }
    ws->control = static_cast<char*>(get(control_bytes()));
    if (batched) {
        ws->lane_vn = static_cast<uint64_t*>(get((size_t)g->n * 16));
        ws->lane_front = static_cast<uint64_t*>(get((size_t)g->n * 8));
        ws->lane_level = static_cast<uint8_t*>(get((size_t)g->n * 64));
    }
    if (!ok) {
        free_workspace(g, ws);
        *st = fail(BFS_ERR_NO_MEMORY, "device memory exhausted while sizing traversal buffers");
        return nullptr;
    }
    ws->ctl = reinterpret_cast<LevelCtl*>(ws->control);
    ws->bar = reinterpret_cast<GridBarrier*>(ws->control + round_up(3 * sizeof(LevelCtl), 128));
    ws->stats = reinterpret_cast<DevStats*>(ws->control + round_up(3 * sizeof(LevelCtl), 128) +
                                            round_up(sizeof(GridBarrier), 128));
    cudaError_t e = cudaMemsetAsync(ws->control, 0, control_bytes(), s);
    if (e != cudaSuccess) {
        free_workspace(g, ws);
        *st = cuda_fail(e, "workspace initialisation");
        return nullptr;
    }
    *st = BFS_OK;
    return ws;
}

static void fill_params(bfs_graph* g, Workspace* ws, TraversalParams& P) {
    std::memset(&P, 0, sizeof(P));
    P.n = g->n;
    P.off = g->d_off;
    P.col = g->d_col;
    P.new2old = g->relabelled ? g->d_new2old : nullptr;
    P.old2new = g->relabelled ? g->d_old2new : nullptr;
    P.t_small = g->t_small;
    P.t_large = g->t_large;
    P.chunk_warp = g->chunk_warp;
    P.chunk_cta = g->chunk_cta;
    P.visited = ws->visited;
    for (int p = 0; p < 2; ++p)
        for (int b = 0; b < kBins; ++b) P.q[p][b] = ws->q[p][b];
    P.ctl = ws->ctl;
    P.bar = ws->bar;
    P.stats = ws->stats;
    P.lane_vn = ws->lane_vn;
    P.lane_front = ws->lane_front;
    P.lane_level = ws->lane_level;
    P.timeout_ns = g->timeout_ns;
    P.debug_stall = g->debug_stall;
    P.use_match_any = g->use_match_any;
    P.hot_words = g->hot_words;
    P.hot_min_edges = g->hot_min_edges;
    // the frontier bitmaps serve bottom-up and bitmap-order levels only; a
    // traversal that runs neither does not maintain them
    const bool need_fb = g->dir_mode != 0 || g->bitmap_div > 0;
    for (int f = 0; f < 3; ++f) P.fb[f] = need_fb ? ws->fb[f] : nullptr;
    P.nnz = g->nnz;
    P.bu_limit = g->relabelled ? g->n_nonzero : g->n;
    P.dir_mode = g->dir_mode;
    P.do_alpha = g->do_alpha;
    P.do_beta = g->do_beta;
    P.dir_override = -1;
    P.bitmap_div = g->bitmap_div;
    // degree-ordered ids put the light bin (deg < t_small) after every
    // heavier vertex; the bins' counts give where it starts
    P.bitmap_from = g->relabelled ? (long long)(g->bin_count[1] + g->bin_count[2]) : 0;
    P.l2_prefetch = g->l2_prefetch;
    P.tma_stage = g->tma_stage;
    P.tma_offset = (int32_t)(((size_t)g->hot_words * 4 + 127) & ~(size_t)127);
    P.timeline = reinterpret_cast<unsigned long long*>(g->timeline);
    P.timeline_cap = g->timeline ? g->timeline_cap : 0;
}

// Dynamic shared memory of the plain kernels: the hot bitmap prefix, then
// (with BFS_OPT_TMA_STAGE) two 1 KB staging buffers per warp.
static size_t plain_smem(const bfs_graph* g) {
    const size_t hot = ((size_t)g->hot_words * 4 + 127) & ~(size_t)127;
    return g->tma_stage ? hot + (size_t)kWarps * 2 * 1024 : (size_t)g->hot_words * 4;
}

static bfs_status grid_size(bfs_graph* g, const void* fn, int32_t* out, size_t smem = 0) {
    int nb = 0;
    // the limit is a property of the kernel, shared by every graph: only raise it
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < smem)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dynamic shared memory size");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kBlock, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (nb < 1) return fail(BFS_ERR_CUDA, "traversal kernel cannot be resident");
    *out = nb * g->ctx->sms;
    return BFS_OK;
}

// The persistent single-source kernel a traversal of g launches: the lean
// build (bfs_kernels_lean.cu) whenever the run asks for none of the paths
// compiled out of it, else the full one.  Both have the same launch bounds
// and shared memory, and the lean one never uses more registers, so the
// full kernel's resident grid is resident for either.
static bool plain_is_lean(const bfs_graph* g) {
    return g->tma_stage == 0 && g->dir_mode == 0 && g->bitmap_div == 0 && g->hot_words == 0 &&
           g->use_match_any == 0 && g->l2_prefetch == 0;
}
static const void* persistent_plain_fn(const bfs_graph* g) {
    return plain_is_lean(g) ? lean::plain_persistent_fn(g->min_blocks)
                            : plain_persistent_fn(g->min_blocks, g->tma_stage != 0);
}

// Plain-kernel grids for the graph's shared-memory setting (both the
// persistent kernel and the host-loop step kernel take the same size).
static bfs_status set_plain_grids(bfs_graph* g) {
    const size_t smem = plain_smem(g);
    int32_t grid2 = 0;
    bfs_status st = grid_size(g, plain_step_fn(g->min_blocks, g->tma_stage != 0), &grid2, smem);
    if (st != BFS_OK) return st;
    return grid_size(g, plain_persistent_fn(g->min_blocks, g->tma_stage != 0), &g->grid_plain, smem);
}

static bfs_status dev_status(int s) {
    switch (s) {
    case kDevOk: return BFS_OK;
    case kDevTimeout: return fail(BFS_ERR_TIMEOUT, "device-side grid barrier wait timed out");
    case kDevDepth: return fail(BFS_ERR_DEPTH_OVERFLOW, "int8 distances: level above 126");
    default: return fail(BFS_ERR_CUDA, "device queue overflow (internal error)");
    }
}

static bfs_status launch_coop(const void* fn, int grid, TraversalParams& P, cudaStream_t s,
                              size_t smem = 0) {
    void* args[] = {&P};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "cooperative launch");
    return BFS_OK;
}

static bfs_status launch_plain_kernel(const void* fn, int grid, TraversalParams& P,
                                      cudaStream_t s, size_t smem = 0) {
    void* args[] = {&P};
    cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return BFS_OK;
}

static bfs_status read_ctl(Workspace* ws, int slot, LevelCtl* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(out, ws->ctl + slot, sizeof(LevelCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "frontier size readback");
    return BFS_OK;
}

static bool ctl_empty(const LevelCtl& c) {
    return (c.packed[0] >> kCountShift) + (c.packed[1] >> kCountShift) +
               (c.packed[2] >> kCountShift) ==
           0;
}

// ------------------------------------------- graph-captured level loop
// One instantiated CUDA graph per graph and kind (single-source, batched):
// init -> seed -> while(cond) { level kernels -> one-CTA step that sets
// cond } [-> emit].  The key is the launch parameters without the per-run
// fields; when a run's key matches, only the seed node's parameters (the
// roots) are updated before the launch, otherwise the graph is rebuilt.
struct GraphLoop {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t seed = nullptr;
    cudaGraphConditionalHandle cond = 0;
    const void* fn = nullptr;
    size_t smem = 0;
    TraversalParams key;
};

void graph_loop_free(GraphLoop*& gl) {
    if (!gl) return;
    if (gl->exec) cudaGraphExecDestroy(gl->exec);
    if (gl->graph) cudaGraphDestroy(gl->graph);
    delete gl;
    gl = nullptr;
}

static TraversalParams graph_key(const TraversalParams& P) {
    TraversalParams k;
    std::memcpy(&k, &P, sizeof(k));
    k.root_caller = 0;
    std::memset(k.roots, 0, sizeof(k.roots));
    k.phase = 0;
    k.level = 0;
    k.graph_cond = 0;
    return k;
}

static cudaError_t add_step_node(cudaGraphNode_t* out, cudaGraph_t gr, const cudaGraphNode_t* dep,
                                 const void* fn, const TraversalParams& P, int phase, int blocks,
                                 size_t smem) {
    TraversalParams Q;
    std::memcpy(&Q, &P, sizeof(Q));
    Q.phase = phase;
    void* args[] = {&Q};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3((unsigned)blocks);
    kp.blockDim = dim3(kBlock);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, gr, dep, dep ? 1 : 0, &kp);
}

static bfs_status launch_graph_loop(GraphLoop*& gl, TraversalParams P, const void* fn, bool batched,
                                    int32_t grid, size_t smem, cudaStream_t s) {
    const TraversalParams key = graph_key(P);
    cudaError_t e = cudaSuccess;
    if (gl && gl->fn == fn && gl->smem == smem && std::memcmp(&gl->key, &key, sizeof(key)) == 0) {
        TraversalParams Q;
        std::memcpy(&Q, &P, sizeof(Q));
        Q.phase = 1;
        Q.graph_cond = gl->cond;
        void* args[] = {&Q};
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void*>(fn);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(kBlock);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = args;
        e = cudaGraphExecKernelNodeSetParams(gl->exec, gl->seed, &kp);
        if (e == cudaSuccess) e = cudaGraphLaunch(gl->exec, s);
        return e == cudaSuccess ? BFS_OK : cuda_fail(e, "graph loop launch");
    }
    graph_loop_free(gl);
    gl = new (std::nothrow) GraphLoop();
    if (!gl) return fail(BFS_ERR_NO_MEMORY, "host allocation failed");
    gl->fn = fn;
    gl->smem = smem;
    std::memcpy(&gl->key, &key, sizeof(key));
    cudaGraphNode_t n_init = nullptr, n_while = nullptr, b1 = nullptr, b2 = nullptr, b3 = nullptr;
    cudaGraphNode_t n_emit = nullptr;
    e = cudaGraphCreate(&gl->graph, 0);
    if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&gl->cond, gl->graph, 1u, cudaGraphCondAssignDefault);
    P.graph_cond = gl->cond;
    if (e == cudaSuccess) e = add_step_node(&n_init, gl->graph, nullptr, fn, P, 0, grid, smem);
    if (e == cudaSuccess) e = add_step_node(&gl->seed, gl->graph, &n_init, fn, P, 1, 1, smem);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = gl->cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&n_while, gl->graph, &gl->seed, nullptr, 1, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (!batched) {
        if (e == cudaSuccess) e = add_step_node(&b1, body, nullptr, fn, P, 5, grid, smem);
        if (e == cudaSuccess) e = add_step_node(&b2, body, &b1, fn, P, 6, 1, smem);
    } else {
        if (e == cudaSuccess) e = add_step_node(&b1, body, nullptr, fn, P, 7, grid, smem);
        if (e == cudaSuccess) e = add_step_node(&b2, body, &b1, fn, P, 8, grid, smem);
        if (e == cudaSuccess) e = add_step_node(&b3, body, &b2, fn, P, 9, 1, smem);
        if (e == cudaSuccess) e = add_step_node(&n_emit, gl->graph, &n_while, fn, P, 4, grid, smem);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gl->exec, gl->graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(gl->exec, s);
    if (e != cudaSuccess) {
        graph_loop_free(gl);
        return cuda_fail(e, "graph loop");
    }
    return BFS_OK;
}

bfs_status run_plain_on(bfs_graph* g, Workspace* ws, int32_t root, int32_t* dist,
                        int32_t* parent, cudaStream_t s, uint32_t flags, int32_t grid) {
    TraversalParams P;
    fill_params(g, ws, P);
    P.dist = dist;
    P.parent = parent;
    P.root_caller = root;
    const size_t smem = plain_smem(g);
    if (flags & BFS_GRAPH_LOOP)
        return launch_graph_loop(g->loop_plain, P, plain_step_fn(g->min_blocks, g->tma_stage != 0),
                                 false, grid > 0 ? grid : g->grid_plain, smem, s);
    if (!(flags & BFS_HOST_LOOP))
        return launch_coop(persistent_plain_fn(g), grid > 0 ? grid : g->grid_plain, P, s, smem);
    // host-driven level loop: init, seed, then one launch per level
    bfs_status st;
    const void* fn = plain_step_fn(g->min_blocks, g->tma_stage != 0);
    P.phase = 0;
    if ((st = launch_plain_kernel(fn, g->grid_plain, P, s, smem)) != BFS_OK) return st;
    P.phase = 1;
    if ((st = launch_plain_kernel(fn, 1, P, s, smem)) != BFS_OK) return st;
    P.phase = 2;
    // the host takes the same direction decisions as the device loop
    LevelCtl c;
    if ((st = read_ctl(ws, 0, &c, s)) != BFS_OK) return st;
    long long seen_edges = 0;
    bool prev_bu = false;
    for (int level = 0;; ++level) {
        long long nf = 0, mf = 0;
        for (int b = 0; b < kBins; ++b) {
            nf += (long long)(c.packed[b] >> kCountShift);
            mf += (long long)(c.packed[b] & kEdgeMask);
        }
        seen_edges += mf;
        const int dir = choose_direction(g->dir_mode, prev_bu, mf, g->nnz - seen_edges, nf, g->n,
                                         g->do_alpha, g->do_beta, g->bitmap_div);
        prev_bu = dir == 2;
        P.level = level;
        P.dir_override = dir;
        TraceRange lv("level", level);
        if ((st = launch_plain_kernel(fn, g->grid_plain, P, s, smem)) != BFS_OK) return st;
        if ((st = read_ctl(ws, (level + 1) % 3, &c, s)) != BFS_OK) return st;
        if (ctl_empty(c)) {
            P.level = level + 1;  // books the last level's discoveries
            return launch_plain_kernel(fn, 1, P, s, smem);
        }
    }
}

bfs_status run_batch_on(bfs_graph* g, Workspace* ws, const int32_t* roots, int32_t k, void* dist,
                        cudaStream_t s, uint32_t flags, int32_t grid) {
    if (grid <= 0) grid = g->grid_batch;
    TraversalParams P;
    fill_params(g, ws, P);
    P.nlanes = k;
    P.dist_int8 = (flags & BFS_DIST_INT8) ? 1 : 0;
    for (int i = 0; i < k; ++i) P.roots[i] = roots[i];
    P.dist = static_cast<int32_t*>(dist);
    if (flags & BFS_GRAPH_LOOP)
        return launch_graph_loop(g->loop_batch, P, batch_step_fn(g->min_blocks), true, grid, 0, s);
    if (!(flags & BFS_HOST_LOOP)) return launch_coop(batch_persistent_fn(g->min_blocks), grid, P, s);
    bfs_status st;
    P.phase = 0;
    if ((st = launch_plain_kernel(batch_step_fn(g->min_blocks), grid, P, s)) != BFS_OK) return st;
    P.phase = 1;
    if ((st = launch_plain_kernel(batch_step_fn(g->min_blocks), 1, P, s)) != BFS_OK) return st;
    for (int level = 0;; ++level) {
        LevelCtl c;
        if ((st = read_ctl(ws, level % 3, &c, s)) != BFS_OK) return st;
        if (ctl_empty(c)) break;
        if (P.dist_int8 && level + 1 > 126)
            return fail(BFS_ERR_DEPTH_OVERFLOW, "int8 distances: level above 126");
        P.level = level;
        P.phase = 2;
        TraceRange lv("level", level);
        if ((st = launch_plain_kernel(batch_step_fn(g->min_blocks), grid, P, s)) != BFS_OK) return st;
        P.phase = 3;
        if ((st = launch_plain_kernel(batch_step_fn(g->min_blocks), grid, P, s)) != BFS_OK) return st;
        LevelCtl nc;
        if ((st = read_ctl(ws, (level + 1) % 3, &nc, s)) != BFS_OK) return st;
        if (nc.new_lanes > 0) {
            const long long lv = level + 2;
            cudaError_t e = cudaMemcpyAsync(&ws->stats->levels, &lv, sizeof(lv),
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "level count");
        }
    }
    P.phase = 4;  // distance rows in the caller's numbering
    return launch_plain_kernel(batch_step_fn(g->min_blocks), grid, P, s);
}

static bfs_status finish(Workspace* ws, cudaStream_t s, bfs_run_stats* out) {
    DevStats h;
    cudaError_t e = cudaMemcpyAsync(&h, ws->stats, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "traversal");
    if (out) {
        out->levels = h.levels;
        out->reached = h.reached;
        out->edges_scanned = h.edges;
        out->status = h.status;
        out->bottom_up_levels = h.bu_levels;
    }
    return dev_status(h.status);
}

bfs_status batch_finish(bfs_graph* g, Workspace* ws, cudaStream_t s, bfs_run_stats* stats) {
    (void)g;
    return finish(ws, s, stats);
}

int32_t plain_grid_of(const bfs_graph* g) { return g->grid_plain; }

bfs_status cta_footprint(const bfs_graph* g, bool batched, CtaFootprint* out) {
    const void* fn = batched ? batch_persistent_fn(g->min_blocks) : persistent_plain_fn(g);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    // registers are allocated per warp in units of 256
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    out->regs = warp_regs * (kBlock / 32);
    out->threads = kBlock;
    out->smem = fa.sharedSizeBytes + (batched ? 0 : plain_smem(g));
    return BFS_OK;
}

static bfs_status ensure_workspace(bfs_graph* g, bool batched, cudaStream_t s, Workspace** out) {
    Workspace*& slot = batched ? g->ws_batch : g->ws_plain;
    if (!slot) {
        bfs_status st;
        slot = make_workspace(g, g->ctx->mem, batched, s, &st);
        if (!slot) return st;
    }
    *out = slot;
    return BFS_OK;
}

}  // namespace bfs

using namespace bfs;

// ============================================================== C ABI

extern "C" {

const char* bfs_last_error(void) { return t_last_error.c_str(); }

int32_t bfs_version(void) { return 100; }

const char* bfs_status_string(bfs_status s) {
    switch (s) {
    case BFS_OK: return "ok";
    case BFS_PENDING: return "pending";
    case BFS_ERR_INVALID_ARG: return "invalid argument";
    case BFS_ERR_INVALID_GRAPH: return "invalid graph";
    case BFS_ERR_ROOT_RANGE: return "root out of range";
    case BFS_ERR_NO_MEMORY: return "out of device memory";
    case BFS_ERR_BUDGET: return "query exceeds the memory budget";
    case BFS_ERR_DEPTH_OVERFLOW: return "depth overflow";
    case BFS_ERR_TIMEOUT: return "device wait timed out";
    case BFS_ERR_CUDA: return "CUDA error";
    case BFS_ERR_UNSUPPORTED: return "unsupported";
    case BFS_ERR_CANCELLED: return "cancelled";
    case BFS_ERR_NOT_FOUND: return "not found";
    default: return "unknown status";
    }
}

bfs_status bfs_context_create(int device, void* arena, size_t arena_bytes, bfs_context** out) {
    if (!out) return fail(BFS_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (arena && arena_bytes < 4096) return fail(BFS_ERR_INVALID_ARG, "arena too small");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(BFS_ERR_INVALID_ARG, "no such device");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
        return cuda_fail(e, "cudaGetDeviceProperties");
    if (!prop.cooperativeLaunch) return fail(BFS_ERR_UNSUPPORTED, "device lacks cooperative launch");
    bfs_context* c = new (std::nothrow) bfs_context();
    if (!c) return fail(BFS_ERR_NO_MEMORY, "host allocation failed");
    c->device = device;
    c->sms = prop.multiProcessorCount;
    c->l2_bytes = prop.l2CacheSize;
    c->mem = new DeviceAllocator(arena, arena_bytes);
    *out = c;
    return BFS_OK;
}

bfs_status bfs_context_destroy(bfs_context* ctx) {
    if (!ctx) return fail(BFS_ERR_INVALID_ARG, "null context");
    delete ctx->mem;
    delete ctx;
    return BFS_OK;
}

bfs_status bfs_context_memory(const bfs_context* ctx, size_t* used, size_t* capacity) {
    if (!ctx) return fail(BFS_ERR_INVALID_ARG, "null context");
    if (used) *used = ctx->mem->used();
    if (capacity) *capacity = ctx->mem->capacity();
    return BFS_OK;
}

static bfs_status compute_bins(bfs_graph* g, cudaStream_t s) {
    unsigned long long* d = static_cast<unsigned long long*>(g->ctx->mem->alloc(8 * 8));
    if (!d) return fail(BFS_ERR_NO_MEMORY, "device memory exhausted (degree histogram)");
    unsigned long long h[8] = {0};
    cudaError_t e = cudaMemsetAsync(d, 0, 8 * 8, s);
    if (e == cudaSuccess)
        e = launch_degree_bins(g->d_off, g->n, g->t_small, g->t_large, d, d + 3, d + 6,
                               g->ctx->sms, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    g->ctx->mem->release(d);
    if (e != cudaSuccess) return cuda_fail(e, "degree histogram");
    for (int b = 0; b < kBins; ++b) {
        g->bin_count[b] = h[b];
        g->bin_edges[b] = h[3 + b];
    }
    g->max_degree = (int64_t)h[6];
    g->n_nonzero = (int64_t)(h[0] + h[1] + h[2]);
    if (g->max_degree > 0x7fffffffll)
        return fail(BFS_ERR_UNSUPPORTED, "a vertex has more than 2^31-1 adjacency entries");
    return BFS_OK;
}

bfs_status bfs_graph_upload(bfs_context* ctx, const int64_t* row_off, const int32_t* col,
                            int64_t n, int64_t nnz, uint32_t flags, void* stream,
                            bfs_graph** out) {
    TraceRange tr("bfs_graph_upload", n);
    if (!ctx || !row_off || !out || (!col && nnz > 0))
        return fail(BFS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n < 1 || nnz < 0) return fail(BFS_ERR_INVALID_ARG, "n must be >= 1 and nnz >= 0");
    if (n > kMaxVertices || nnz > kMaxEdges)
        return fail(BFS_ERR_UNSUPPORTED, "graph exceeds 2^30-1 vertices or 2^34-1 entries");
    if (flags & ~(BFS_UPLOAD_DEVICE_PTRS | BFS_UPLOAD_NO_RELABEL))
        return fail(BFS_ERR_INVALID_ARG, "unknown upload flag");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const bool dev_src = (flags & BFS_UPLOAD_DEVICE_PTRS) != 0;
    if (!dev_src) {
        if (row_off[0] != 0 || row_off[n] != nnz)
            return fail(BFS_ERR_INVALID_GRAPH, "row_off[0] must be 0 and row_off[n] must be nnz");
    }
    bfs_graph* g = new (std::nothrow) bfs_graph();
    if (!g) return fail(BFS_ERR_NO_MEMORY, "host allocation failed");
    g->ctx = ctx;
    g->n = n;
    g->nnz = nnz;
    DeviceAllocator* m = ctx->mem;
    const size_t off_bytes = (size_t)(n + 1) * 8;
    const size_t col_bytes = (size_t)(nnz + 16) * 4;  // padded for 16-byte rounded reads
    g->d_off = static_cast<int64_t*>(m->alloc(off_bytes));
    g->d_col = static_cast<int32_t*>(m->alloc(col_bytes));
    int* d_flags = static_cast<int*>(m->alloc(16));
    auto cleanup = [&](bfs_status st) {
        m->release(d_flags);
        bfs_graph_free(g);
        return st;
    };
    if (!g->d_off || !g->d_col || !d_flags)
        return cleanup(fail(BFS_ERR_NO_MEMORY, "device memory exhausted (graph)"));
    g->graph_bytes = round_up(off_bytes, kAlign) + round_up(col_bytes, kAlign);
    const cudaMemcpyKind kind = dev_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = cudaMemcpyAsync(g->d_off, row_off, off_bytes, kind, s);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(g->d_col, col, (size_t)nnz * 4, kind, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_col + nnz, 0, 16 * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flags, 0, 16, s);
    if (e == cudaSuccess) e = launch_csr_check(g->d_off, g->d_col, n, nnz, d_flags, ctx->sms, s);
    int h_flags = 0;
    int64_t ends[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flags, d_flags, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[0], g->d_off, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], g->d_off + n, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "graph upload"));
    if (ends[0] != 0 || ends[1] != nnz)
        return cleanup(fail(BFS_ERR_INVALID_GRAPH, "row_off[0] must be 0 and row_off[n] must be nnz"));
    if (h_flags & 2) return cleanup(fail(BFS_ERR_INVALID_GRAPH, "row offsets decrease"));
    if (h_flags & 1) return cleanup(fail(BFS_ERR_INVALID_GRAPH, "column index out of range"));
    {
        // symmetric graphs (each edge stored both ways) may run bottom-up levels
        unsigned long long h[2] = {0, 0};
        unsigned long long* d_sums = reinterpret_cast<unsigned long long*>(d_flags);
        e = cudaMemsetAsync(d_sums, 0, 16, s);
        if (e == cudaSuccess) e = launch_symmetry_hash(g->d_off, g->d_col, n, d_sums, ctx->sms, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_sums, 16, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "symmetry test"));
        g->symmetric = h[0] == h[1];
    }
    m->release(d_flags);
    d_flags = nullptr;
    if (!(flags & BFS_UPLOAD_NO_RELABEL)) {
        // degree-ordered renumbering on the device; the uploaded copy is
        // replaced by the renumbered one
        int64_t* n_off = static_cast<int64_t*>(m->alloc(off_bytes));
        int32_t* n_col = static_cast<int32_t*>(m->alloc(col_bytes));
        g->d_new2old = static_cast<int32_t*>(m->alloc((size_t)n * 4));
        g->d_old2new = static_cast<int32_t*>(m->alloc((size_t)n * 4));
        void* scratch = m->alloc(relabel_scratch_bytes(n));
        if (!n_off || !n_col || !g->d_new2old || !g->d_old2new || !scratch) {
            m->release(n_off);
            m->release(n_col);
            m->release(scratch);
            return cleanup(fail(BFS_ERR_NO_MEMORY, "device memory exhausted (renumbering)"));
        }
        e = relabel_graph(g->d_off, g->d_col, n, nnz, ctx->sms, g->d_new2old, g->d_old2new, n_off,
                          n_col, scratch, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(n_col + nnz, 0, 16 * 4, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        m->release(scratch);
        if (e != cudaSuccess) {
            m->release(n_off);
            m->release(n_col);
            return cleanup(cuda_fail(e, "renumbering"));
        }
        m->release(g->d_off);
        m->release(g->d_col);
        g->d_off = n_off;
        g->d_col = n_col;
        g->relabelled = true;
        g->graph_bytes += 2 * round_up((size_t)n * 4, kAlign);
    }
    bfs_status st = compute_bins(g, s);
    if (st != BFS_OK) return cleanup(st);
    // the shared-memory copy of the hot bitmap prefix is off by default: on
    // GB300 the degree-ordered bitmap's hot words already hit in L1, and the
    // shared memory it takes shrinks that L1 (measured slower)
    g->hot_words = 0;
    if ((st = set_plain_grids(g)) != BFS_OK) return cleanup(st);
    if ((st = grid_size(g, batch_persistent_fn(g->min_blocks), &g->grid_batch)) != BFS_OK) return cleanup(st);
    Workspace* ws = nullptr;
    if ((st = ensure_workspace(g, false, s, &ws)) != BFS_OK) return cleanup(st);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "graph upload"));
    *out = g;
    return BFS_OK;
}

bfs_status bfs_graph_free(bfs_graph* g) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    cudaSetDevice(g->ctx->device);
    cudaDeviceSynchronize();
    DeviceAllocator* m = g->ctx->mem;
    graph_loop_free(g->loop_plain);
    graph_loop_free(g->loop_batch);
    free_workspace(g, g->ws_plain);
    free_workspace(g, g->ws_batch);
    m->release(g->d_off);
    m->release(g->d_col);
    m->release(g->d_new2old);
    m->release(g->d_old2new);
    delete g;
    return BFS_OK;
}

bfs_status bfs_graph_get_info(const bfs_graph* g, bfs_graph_info* out) {
    if (!g || !out) return fail(BFS_ERR_INVALID_ARG, "null argument");
    out->n = g->n;
    out->nnz = g->nnz;
    out->max_degree = g->max_degree;
    out->t_small = g->t_small;
    out->t_large = g->t_large;
    out->chunk_warp = g->chunk_warp;
    out->chunk_cta = g->chunk_cta;
    out->relabelled = g->relabelled ? 1 : 0;
    out->grid_blocks = g->grid_plain;
    out->device_bytes = g->graph_bytes + (g->ws_plain ? g->ws_plain->bytes : 0) +
                        (g->ws_batch ? g->ws_batch->bytes : 0);
    return BFS_OK;
}

bfs_status bfs_graph_set_bins(bfs_graph* g, int32_t t_small, int32_t t_large, int32_t chunk_warp,
                              int32_t chunk_cta) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    auto pow2 = [](int32_t x) { return x > 0 && (x & (x - 1)) == 0; };
    if (t_small < 1 || t_large <= t_small || t_small > (1 << 20) || chunk_warp < 128 ||
        chunk_warp > (1 << 24) || !pow2(chunk_warp) || chunk_cta < 1024 ||
        chunk_cta > (1 << 24) || !pow2(chunk_cta))
        return fail(BFS_ERR_INVALID_ARG,
                    "bad bin thresholds or chunk sizes (chunks: powers of two, warp >= 128, "
                    "CTA >= 1024, both <= 2^24)");
    std::lock_guard<std::mutex> lk(g->mu);
    cudaSetDevice(g->ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before re-binning");
    free_workspace(g, g->ws_plain);
    free_workspace(g, g->ws_batch);
    g->ws_plain = g->ws_batch = nullptr;
    g->t_small = t_small;
    g->t_large = t_large;
    g->chunk_warp = chunk_warp;
    g->chunk_cta = chunk_cta;
    bfs_status st = compute_bins(g, nullptr);
    if (st != BFS_OK) return st;
    Workspace* ws;
    if ((st = ensure_workspace(g, false, nullptr, &ws)) != BFS_OK) return st;
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? BFS_OK : cuda_fail(e, "re-binning");
}

bfs_status bfs_run(bfs_graph* g, int32_t root, int32_t* dist, int32_t* parent, void* stream,
                   uint32_t flags) {
    TraceRange tr("bfs_run", root);
    if (!g || !dist) return fail(BFS_ERR_INVALID_ARG, "null graph or dist");
    if (flags & ~(BFS_OUT_HOST | BFS_HOST_LOOP | BFS_GRAPH_LOOP | BFS_DIST_INT8))
        return fail(BFS_ERR_INVALID_ARG, "unknown flag");
    if ((flags & BFS_HOST_LOOP) && (flags & BFS_GRAPH_LOOP))
        return fail(BFS_ERR_INVALID_ARG, "BFS_HOST_LOOP and BFS_GRAPH_LOOP are exclusive");
    if (root < 0 || root >= g->n) return fail(BFS_ERR_ROOT_RANGE, "root out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaSetDevice(g->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Workspace* ws = nullptr;
    bfs_status st = ensure_workspace(g, false, s, &ws);
    if (st != BFS_OK) return st;
    const bool host = (flags & BFS_OUT_HOST) != 0;
    const bool int8 = (flags & BFS_DIST_INT8) != 0;
    // int32 distances go to the caller's buffer, or to staging when they are
    // copied to the host or turned into int8 rows afterwards
    int32_t* d_dist = dist;
    int32_t* d_parent = parent;
    int8_t* d_dist8 = int8 && !host ? reinterpret_cast<int8_t*>(dist) : nullptr;
    if (host || int8) {
        if (!ws->dist_scratch) ws->dist_scratch = static_cast<int32_t*>(g->ctx->mem->alloc(g->n * 4));
        if (!ws->dist_scratch) return fail(BFS_ERR_NO_MEMORY, "device memory exhausted (output staging)");
        d_dist = ws->dist_scratch;
    }
    if (host) {
        if (parent && !ws->parent_scratch)
            ws->parent_scratch = static_cast<int32_t*>(g->ctx->mem->alloc(g->n * 4));
        if (int8 && !ws->dist8_scratch)
            ws->dist8_scratch = static_cast<int8_t*>(g->ctx->mem->alloc(g->n + 16));
        if ((parent && !ws->parent_scratch) || (int8 && !ws->dist8_scratch))
            return fail(BFS_ERR_NO_MEMORY, "device memory exhausted (output staging)");
        d_parent = parent ? ws->parent_scratch : nullptr;
        if (int8) d_dist8 = ws->dist8_scratch;
    }
    if ((st = run_plain_on(g, ws, root, d_dist, d_parent, s, flags & ~BFS_DIST_INT8, 0)) != BFS_OK)
        return st;
    if (int8) {
        e = launch_dist_to_int8(d_dist, d_dist8, g->n, ws->stats, g->ctx->sms, s);
        if (e != cudaSuccess) return cuda_fail(e, "int8 rows");
    }
    if (!host) return BFS_OK;
    if (int8) e = cudaMemcpyAsync(dist, d_dist8, g->n, cudaMemcpyDeviceToHost, s);
    else e = cudaMemcpyAsync(dist, d_dist, g->n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && parent)
        e = cudaMemcpyAsync(parent, d_parent, g->n * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    return finish(ws, s, nullptr);
}

bfs_status bfs_graph_sync(bfs_graph* g, void* stream, bfs_run_stats* stats) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    std::lock_guard<std::mutex> lk(g->mu);
    cudaSetDevice(g->ctx->device);
    if (!g->ws_plain) return fail(BFS_ERR_NOT_FOUND, "no traversal has run");
    return finish(g->ws_plain, static_cast<cudaStream_t>(stream), stats);
}

bfs_status bfs_run_batch(bfs_graph* g, const int32_t* roots, int32_t k, void* dist, void* stream,
                         uint32_t flags) {
    TraceRange tr("bfs_run_batch", k);
    if (!g || !roots || !dist) return fail(BFS_ERR_INVALID_ARG, "null argument");
    if (k < 1 || k > 64) return fail(BFS_ERR_INVALID_ARG, "k must be in 1..64");
    if (flags & ~(BFS_OUT_HOST | BFS_DIST_INT8 | BFS_HOST_LOOP | BFS_GRAPH_LOOP))
        return fail(BFS_ERR_INVALID_ARG, "unknown flag");
    if ((flags & BFS_HOST_LOOP) && (flags & BFS_GRAPH_LOOP))
        return fail(BFS_ERR_INVALID_ARG, "BFS_HOST_LOOP and BFS_GRAPH_LOOP are exclusive");
    for (int i = 0; i < k; ++i)
        if (roots[i] < 0 || roots[i] >= g->n) return fail(BFS_ERR_ROOT_RANGE, "root out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaSetDevice(g->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    Workspace* ws = nullptr;
    bfs_status st = ensure_workspace(g, true, s, &ws);
    if (st != BFS_OK) return st;
    const size_t elt = (flags & BFS_DIST_INT8) ? 1 : 4;
    const size_t bytes = (size_t)k * g->n * elt;
    void* d_dist = dist;
    const bool host = (flags & BFS_OUT_HOST) != 0;
    if (host) {
        if (!ws->batch_dist_scratch)
            ws->batch_dist_scratch = g->ctx->mem->alloc((size_t)64 * g->n * 4);
        if (!ws->batch_dist_scratch)
            return fail(BFS_ERR_NO_MEMORY, "device memory exhausted (output staging)");
        d_dist = ws->batch_dist_scratch;
    }
    if ((st = run_batch_on(g, ws, roots, k, d_dist, s, flags, 0)) != BFS_OK) return st;
    if (!host) return BFS_OK;
    e = cudaMemcpyAsync(dist, d_dist, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    return finish(ws, s, nullptr);
}

bfs_status bfs_batch_sync(bfs_graph* g, void* stream, bfs_run_stats* stats) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    std::lock_guard<std::mutex> lk(g->mu);
    cudaSetDevice(g->ctx->device);
    if (!g->ws_batch) return fail(BFS_ERR_NOT_FOUND, "no batched traversal has run");
    return finish(g->ws_batch, static_cast<cudaStream_t>(stream), stats);
}

bfs_status bfs_graph_set_option(bfs_graph* g, int32_t option, int64_t value) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    std::lock_guard<std::mutex> lk(g->mu);
    switch (option) {
    case BFS_OPT_WARP_AGGREGATE:
        if (value != 0 && value != 1) return fail(BFS_ERR_INVALID_ARG, "value must be 0 or 1");
        g->use_match_any = (int32_t)value;
        return BFS_OK;
    case BFS_OPT_TIMEOUT_NS:
        if (value <= 0) return fail(BFS_ERR_INVALID_ARG, "timeout must be positive");
        g->timeout_ns = value;
        return BFS_OK;
    case BFS_OPT_CTAS_PER_SM: {
        if (value < 2 || value > 4) return fail(BFS_ERR_INVALID_ARG, "value must be 2, 3 or 4");
        g->min_blocks = (int32_t)value;
        bfs_status st = set_plain_grids(g);
        if (st == BFS_OK) st = grid_size(g, batch_persistent_fn(g->min_blocks), &g->grid_batch);
        return st;
    }
    case BFS_OPT_HOT_WORDS: {
        if (value < 0 || value > 40960 || value % 4) return fail(BFS_ERR_INVALID_ARG, "hot words must be a multiple of 4 in [0, 40960]");
        const int32_t old = g->hot_words;
        g->hot_words = (int32_t)value;
        bfs_status st = set_plain_grids(g);
        if (st != BFS_OK) {
            g->hot_words = old;
            set_plain_grids(g);
        }
        return st;
    }
    case BFS_OPT_HOT_MIN_EDGES:
        if (value < 0) return fail(BFS_ERR_INVALID_ARG, "must be >= 0");
        g->hot_min_edges = value;
        return BFS_OK;
    case BFS_OPT_DIRECTION:
        if (value < 0 || value > 2) return fail(BFS_ERR_INVALID_ARG, "direction must be 0, 1 or 2");
        if (value != 0 && !g->symmetric)
            return fail(BFS_ERR_UNSUPPORTED,
                        "bottom-up levels need a symmetric graph (every edge stored both ways)");
        g->dir_mode = (int32_t)value;
        return BFS_OK;
    case BFS_OPT_L2_PREFETCH:
        if (value < 0 || value > 1) return fail(BFS_ERR_INVALID_ARG, "must be 0 or 1");
        g->l2_prefetch = (int32_t)value;
        return BFS_OK;
    case BFS_OPT_TMA_STAGE: {
        if (value < 0 || value > 1) return fail(BFS_ERR_INVALID_ARG, "must be 0 or 1");
        const int32_t old = g->tma_stage;
        g->tma_stage = (int32_t)value;
        bfs_status st = set_plain_grids(g);
        if (st != BFS_OK) {
            g->tma_stage = old;
            set_plain_grids(g);
        }
        return st;
    }
    case BFS_OPT_BITMAP_FRONTIER:
        if (value < 0 || value > (1 << 20)) return fail(BFS_ERR_INVALID_ARG, "must be in [0, 2^20]");
        g->bitmap_div = (int32_t)value;
        return BFS_OK;
    case BFS_OPT_DO_ALPHA:
    case BFS_OPT_DO_BETA:
        if (value < 1 || value > (1 << 20)) return fail(BFS_ERR_INVALID_ARG, "must be in [1, 2^20]");
        (option == BFS_OPT_DO_ALPHA ? g->do_alpha : g->do_beta) = (int32_t)value;
        return BFS_OK;
    default: return fail(BFS_ERR_INVALID_ARG, "unknown option");
    }
}

bfs_status bfs_debug_set_barrier_test(bfs_graph* g, int32_t stall, int64_t timeout_ns) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    std::lock_guard<std::mutex> lk(g->mu);
    g->debug_stall = stall ? 1 : 0;
    g->timeout_ns = timeout_ns > 0 ? timeout_ns : 2000000000ll;
    return BFS_OK;
}

bfs_status bfs_debug_set_timeline(bfs_graph* g, uint64_t* d_stamps, int32_t cap) {
    if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
    if (d_stamps && cap < 3) return fail(BFS_ERR_INVALID_ARG, "a timeline needs at least 3 entries");
    std::lock_guard<std::mutex> lk(g->mu);
    g->timeline = d_stamps;
    g->timeline_cap = d_stamps ? cap : 0;
    return BFS_OK;
}

}  // extern "C"
