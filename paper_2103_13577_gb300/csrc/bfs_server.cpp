// bfs_server.cpp -- continuous-batching query server behind bfs_submit /
// bfs_poll.
//
// One dispatcher thread owns every launch.  Queries wait in a FIFO per
// graph.  Whenever a stream slot is free and the server's device arena
// (its memory budget) can hold a launch's traversal buffers and distance
// rows, the dispatcher takes up to 64 waiting queries of one graph (graphs
// served round robin) and runs them on that slot's stream -- as one batched
// traversal, or, when few are waiting, as that many single-source
// traversals (the cut-over is calibrated per graph when it is added) --
// enqueues the copies of each query's row into the caller's buffer, and
// records an event.  Completed events release the memory, which admits
// the next launch -- so queries that arrive while others are on the GPU
// join the next launch on a free slot, and launches on different slots
// overlap on the device: a launch takes as many CTAs per SM as fit next to
// the CTAs of the launches whose kernels are still running (registers,
// threads, shared memory), so every persistent grid is resident at once
// and none waits on another's SMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bfs_runtime.h"

namespace bfs {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Query {
    bfs_ticket ticket = 0;
    int32_t graph_id = 0;
    int32_t root = 0;
    void* dist_out = nullptr;    // int32[n], or int8[n] for an int8 query
    bool int8 = false;
    bfs_status status = BFS_PENDING;
    int64_t submit_ns = 0, launch_ns = 0, done_ns = 0;
};

struct Launch {
    int slot = -1;
    int32_t graph_id = 0;
    bool plain = false;      // k single-source traversals instead of one batched launch
    int ctas_per_sm = 0;     // resident CTAs of its kernel on every SM
    CtaFootprint cta;        // what one of them holds
    Workspace* ws = nullptr;
    void* d_dist = nullptr;
    void* d_dist8 = nullptr;   // int8 rows of a single-source launch of int8 queries
    std::vector<std::shared_ptr<Query>> lanes;
    cudaEvent_t done = nullptr;
};

// Per-graph launch policy: up to plain_max waiting queries are served as
// that many single-source traversals (their mean completion time is no
// later than one batched launch's, whose cost barely depends on how many
// lanes it carries); more go batched.
struct GraphPolicy {
    int32_t plain_max = 0;
    double plain_ms = 0.0, batch_ms = 0.0;
};

struct SlotState {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;     // the launch's kernels and result copies are done
    cudaEvent_t kevent = nullptr;    // its kernels are done (the SMs are free again)
    bool busy = false;
};

}  // namespace bfs

using namespace bfs;

struct bfs_server {
    bfs_context* ctx = nullptr;
    size_t budget = 0;
    void* arena = nullptr;
    DeviceAllocator* mem = nullptr;
    std::vector<bfs_graph*> graphs;
    std::vector<GraphPolicy> policy;
    std::vector<std::deque<std::shared_ptr<Query>>> pending;  // [2 graph + int8]: FIFOs
    std::unordered_map<bfs_ticket, std::shared_ptr<Query>> tickets;
    std::vector<SlotState> slots;
    std::vector<Launch> inflight;
    std::mutex mu;
    std::condition_variable cv_work;   // wakes the dispatcher
    std::condition_variable cv_done;   // wakes waiters
    std::thread dispatcher;
    bool stop = false;
    bfs_ticket next_ticket = 1;
    size_t rr = 0;
    bfs_server_stats stats{};
    size_t inflight_bytes = 0;
    // one SM's resources: launches in flight together must fit in them
    // side by side, or their persistent grids could wait on each other
    int sm_regs = 0, sm_threads = 0;
    size_t sm_smem = 0;
};

namespace bfs {

static size_t launch_bytes(const bfs_graph* g, int k) {
    return std::min(workspace_bytes(g, true, k), workspace_bytes(g, false, k)) + 256 * 32 +
           (size_t)k * g->n * 4 + 4096;
}

// Runs with s->mu held.  Returns true when something was launched.
static bool try_launch(bfs_server* s) {
    int free_slot = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].busy) {
            free_slot = (int)i;
            break;
        }
    if (free_slot < 0) return false;
    const size_t nq = s->pending.size();   // two per graph: int32 and int8 rows
    for (size_t t = 0; t < nq; ++t) {
        const size_t qi = (s->rr + t) % nq;
        const size_t gid = qi / 2;
        const bool int8 = (qi & 1) != 0;
        auto& q = s->pending[qi];
        if (q.empty()) continue;
        bfs_graph* g = s->graphs[gid];
        const int k = (int)std::min<size_t>(64, q.size());
        const bool plain = k <= s->policy[gid].plain_max;
        SlotState& sl = s->slots[free_slot];
        bfs_status st = BFS_OK;
        cudaSetDevice(s->ctx->device);
        // A cooperative launch is only guaranteed to be resident by itself.
        // Each launch takes as many CTAs per SM as fit next to the CTAs of
        // the launches whose kernels are still running (up to its own full
        // grid), so every persistent grid is resident at once: two launches
        // that each got part of their grid would wait on each other's SMs at
        // their grid barriers.  None fits: wait for a kernel to finish.
        CtaFootprint fp;
        if (cta_footprint(g, !plain, &fp) != BFS_OK) continue;
        long long regs = 0, threads = 0;
        size_t smem = 0;
        for (const Launch& o : s->inflight) {
            // a launch whose kernels are done holds no SM resources while
            // its result copies run
            if (cudaEventQuery(s->slots[o.slot].kevent) == cudaSuccess) continue;
            cudaGetLastError();
            regs += (long long)o.ctas_per_sm * o.cta.regs;
            threads += (long long)o.ctas_per_sm * o.cta.threads;
            smem += (size_t)o.ctas_per_sm * o.cta.smem;
        }
        const int32_t full = plain ? plain_grid_of(g) : g->grid_batch;
        long long fit = (full + s->ctx->sms - 1) / s->ctx->sms;
        fit = std::min(fit, (s->sm_regs - regs) / std::max(1, fp.regs));
        fit = std::min(fit, (s->sm_threads - threads) / std::max(1, fp.threads));
        if (fp.smem > 0) fit = std::min(fit, (long long)((s->sm_smem - std::min(smem, s->sm_smem)) / fp.smem));
        if (fit < 1) continue;
        Workspace* ws = make_workspace(g, s->mem, !plain, sl.stream, &st);
        // distance rows: int32 (single-source runs, or an int32 batch), int8
        // for a batch of int8 queries; single-source int8 queries also get
        // int8 rows converted from the int32 ones
        const size_t rows = (size_t)k * g->n;
        void* d_dist = ws ? s->mem->alloc(int8 && !plain ? rows + 16 : rows * 4) : nullptr;
        void* d_dist8 = (ws && int8 && plain) ? s->mem->alloc(rows + 16) : nullptr;
        if (!ws || !d_dist || (int8 && plain && !d_dist8)) {
            if (ws) free_workspace(g, ws);
            s->mem->release(d_dist);
            s->mem->release(d_dist8);
            continue;  // does not fit now; another queue might, or wait for completions
        }
        TraceRange tr("server_launch", k);
        Launch L;
        L.slot = free_slot;
        L.graph_id = (int32_t)gid;
        L.ws = ws;
        L.d_dist = d_dist;
        L.d_dist8 = d_dist8;
        std::vector<int32_t> roots;
        const int64_t t_launch = now_ns();
        for (int i = 0; i < k; ++i) {
            L.lanes.push_back(q.front());
            roots.push_back(q.front()->root);
            q.front()->launch_ns = t_launch;
            q.pop_front();
        }
        L.plain = plain;
        L.cta = fp;
        const int32_t grid = std::min<int32_t>(full, (int32_t)fit * s->ctx->sms);
        L.ctas_per_sm = (int)fit;
        if (plain) {
            for (int i = 0; i < k && st == BFS_OK; ++i)
                st = run_plain_on(g, ws, roots[i], static_cast<int32_t*>(d_dist) + (size_t)i * g->n,
                                  nullptr, sl.stream, 0, grid);
            if (st == BFS_OK && int8) {
                cudaError_t e = launch_dist_to_int8(static_cast<int32_t*>(d_dist),
                                                    static_cast<int8_t*>(d_dist8), (long long)rows,
                                                    ws->stats, s->ctx->sms, sl.stream);
                if (e != cudaSuccess) st = cuda_fail(e, "int8 rows");
            }
        } else {
            st = run_batch_on(g, ws, roots.data(), k, d_dist, sl.stream, int8 ? BFS_DIST_INT8 : 0,
                              grid);
        }
        if (st == BFS_OK) {
            cudaError_t e = cudaEventRecord(sl.kevent, sl.stream);
            if (e != cudaSuccess) st = cuda_fail(e, "event record");
        }
        if (st == BFS_OK) {
            const char* src = static_cast<const char*>(int8 ? (plain ? d_dist8 : d_dist) : d_dist);
            const size_t row = (size_t)g->n * (int8 ? 1 : 4);
            for (int i = 0; i < k; ++i) {
                cudaError_t e = cudaMemcpyAsync(L.lanes[i]->dist_out, src + (size_t)i * row, row,
                                                cudaMemcpyDeviceToHost, sl.stream);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "result copy");
                    break;
                }
            }
        }
        if (st == BFS_OK) {
            cudaError_t e = cudaEventRecord(sl.event, sl.stream);
            if (e != cudaSuccess) st = cuda_fail(e, "event record");
        }
        if (st != BFS_OK) {
            cudaStreamSynchronize(sl.stream);
            for (auto& qq : L.lanes) qq->status = st;
            s->stats.failed += k;
            free_workspace(g, ws);
            s->mem->release(d_dist);
            s->mem->release(d_dist8);
            s->cv_done.notify_all();
            return true;
        }
        L.done = sl.event;
        sl.busy = true;
        s->stats.launches += 1;
        s->stats.lanes += k;
        s->inflight_bytes = s->mem->used();
        s->stats.max_inflight_bytes =
            std::max<int64_t>(s->stats.max_inflight_bytes, (int64_t)s->inflight_bytes);
        s->inflight.push_back(std::move(L));
        s->rr = (qi + 1) % nq;
        return true;
    }
    return false;
}

// Runs with s->mu held.  Retires finished launches; returns how many.
static int reap(bfs_server* s, bool block) {
    int n = 0;
    for (size_t i = 0; i < s->inflight.size();) {
        Launch& L = s->inflight[i];
        cudaError_t e = block ? cudaEventSynchronize(L.done) : cudaEventQuery(L.done);
        if (e == cudaErrorNotReady) {
            ++i;
            continue;
        }
        bfs_status st = BFS_OK;
        if (e != cudaSuccess) st = cuda_fail(e, "batched traversal");
        if (st == BFS_OK) st = batch_finish(s->graphs[L.graph_id], L.ws, s->slots[L.slot].stream, nullptr);
        const int64_t t_done = now_ns();
        for (auto& q : L.lanes) {
            q->status = st;
            q->done_ns = t_done;
        }
        if (st == BFS_OK) s->stats.completed += (int64_t)L.lanes.size();
        else s->stats.failed += (int64_t)L.lanes.size();
        free_workspace(s->graphs[L.graph_id], L.ws);
        s->mem->release(L.d_dist);
        s->mem->release(L.d_dist8);
        s->slots[L.slot].busy = false;
        s->inflight.erase(s->inflight.begin() + (long)i);
        ++n;
    }
    if (n) s->cv_done.notify_all();
    return n;
}

static void dispatcher_main(bfs_server* s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progressed = reap(s, false) > 0;
        while (!s->stop && try_launch(s)) progressed = true;
        bool waiting = false;
        for (auto& q : s->pending)
            if (!q.empty()) waiting = true;
        if (s->stop && s->inflight.empty()) break;
        if (!s->inflight.empty()) {
            // poll completions without holding the lock for long
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(progressed ? 0 : 20));
            lk.lock();
        } else if (!waiting) {
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                for (auto& q : s->pending)
                    if (!q.empty()) return true;
                return false;
            });
        } else if (!progressed) {
            // queries wait but nothing fits and nothing is in flight: they can never run
            for (auto& fifo : s->pending) {
                for (auto& q : fifo) {
                    q->status = BFS_ERR_BUDGET;
                    s->stats.failed += 1;
                }
                fifo.clear();
            }
            s->cv_done.notify_all();
        }
    }
}

}  // namespace bfs

extern "C" {

bfs_status bfs_server_create(bfs_context* ctx, size_t memory_budget, int32_t num_streams,
                             bfs_server** out) {
    if (!ctx || !out) {
        set_error("null argument");
        return BFS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (num_streams < 1 || num_streams > 16 || memory_budget < (1u << 20)) {
        set_error("num_streams must be 1..16 and the budget at least 1 MiB");
        return BFS_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    bfs_server* s = new bfs_server();
    s->ctx = ctx;
    s->budget = memory_budget;
    s->arena = ctx->mem->alloc(memory_budget);
    if (!s->arena) {
        delete s;
        set_error("cannot reserve the server's memory budget on the device");
        return BFS_ERR_NO_MEMORY;
    }
    s->mem = new DeviceAllocator(s->arena, memory_budget);
    int regs = 0, threads = 0, smem = 0;
    e = cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    if (e != cudaSuccess) {
        bfs_status st = cuda_fail(e, "device attributes");
        delete s->mem;
        ctx->mem->release(s->arena);
        delete s;
        return st;
    }
    s->sm_regs = regs;
    s->sm_threads = threads;
    s->sm_smem = (size_t)smem;
    s->slots.resize((size_t)num_streams);
    for (auto& sl : s->slots) {
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.kevent, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            bfs_status st = cuda_fail(e, "stream creation");
            for (auto& x : s->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.event) cudaEventDestroy(x.event);
                if (x.kevent) cudaEventDestroy(x.kevent);
            }
            delete s->mem;
            ctx->mem->release(s->arena);
            delete s;
            return st;
        }
    }
    s->dispatcher = std::thread(dispatcher_main, s);
    *out = s;
    return BFS_OK;
}

bfs_status bfs_server_add_graph(bfs_server* s, bfs_graph* g, int32_t* graph_id) {
    if (!s || !g || !graph_id) {
        set_error("null argument");
        return BFS_ERR_INVALID_ARG;
    }
    // calibrate the launch policy: one single-source run and one 64-lane
    // batched run of the same root, each timed on a scratch stream
    GraphPolicy pol;
    {
        cudaSetDevice(s->ctx->device);
        bfs_status st = BFS_OK;
        Workspace* wp = make_workspace(g, s->ctx->mem, false, nullptr, &st);
        Workspace* wb = wp ? make_workspace(g, s->ctx->mem, true, nullptr, &st) : nullptr;
        void* d = wb ? s->ctx->mem->alloc((size_t)64 * g->n * 4) : nullptr;
        if (!wp || !wb || !d) {
            if (wp) free_workspace(g, wp);
            if (wb) free_workspace(g, wb);
            set_error("server: device memory exhausted while calibrating a graph");
            return BFS_ERR_NO_MEMORY;
        }
        int32_t root = 0;
        for (; root < g->n; ++root) {  // a vertex with out-edges (first in degree order)
            int64_t o[2];
            if (cudaMemcpy(o, g->d_off + root, 16, cudaMemcpyDeviceToHost) != cudaSuccess) break;
            if (o[1] > o[0]) break;
        }
        if (root >= g->n) root = 0;
        std::vector<int32_t> roots(64, root);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float tp = 0.f, tb = 0.f;
        for (int rep = 0; rep < 2 && st == BFS_OK; ++rep) {
            cudaEventRecord(e0, nullptr);
            st = run_plain_on(g, wp, root, static_cast<int32_t*>(d), nullptr, nullptr, 0, 0);
            cudaEventRecord(e1, nullptr);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&tp, e0, e1);
            if (st != BFS_OK) break;
            cudaEventRecord(e0, nullptr);
            st = run_batch_on(g, wb, roots.data(), 64, d, nullptr, 0, 0);
            cudaEventRecord(e1, nullptr);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&tb, e0, e1);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaDeviceSynchronize();
        s->ctx->mem->release(d);
        free_workspace(g, wp);
        free_workspace(g, wb);
        if (st != BFS_OK) return st;
        pol.plain_ms = tp;
        pol.batch_ms = tb;
        // k waiting queries run one by one complete on average after
        // tp (k + 1) / 2, batched after tb: single-source runs while that is
        // no later (the batched launch wins once queues are long)
        pol.plain_max = tp > 0.f ? std::min(63, std::max(0, (int)(2.f * tb / tp) - 1)) : 0;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->graphs.push_back(g);
    s->policy.push_back(pol);
    s->pending.emplace_back();   // int32 rows
    s->pending.emplace_back();   // int8 rows
    *graph_id = (int32_t)s->graphs.size() - 1;
    return BFS_OK;
}

bfs_status bfs_submit_rows(bfs_server* s, int32_t graph_id, int32_t root, void* dist_out,
                           uint32_t flags, bfs_ticket* ticket) {
    if (!s || !dist_out || !ticket) {
        set_error("null argument");
        return BFS_ERR_INVALID_ARG;
    }
    if (flags & ~BFS_DIST_INT8) {
        set_error("unknown flag");
        return BFS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (graph_id < 0 || (size_t)graph_id >= s->graphs.size()) {
        set_error("unknown graph id");
        return BFS_ERR_NOT_FOUND;
    }
    bfs_graph* g = s->graphs[(size_t)graph_id];
    if (root < 0 || root >= g->n) {
        set_error("root out of range");
        return BFS_ERR_ROOT_RANGE;
    }
    if (s->stop) {
        set_error("server is shutting down");
        return BFS_ERR_CANCELLED;
    }
    if (launch_bytes(g, 1) > s->budget) {
        set_error("one query on this graph needs more device memory than the budget");
        return BFS_ERR_BUDGET;
    }
    auto q = std::make_shared<Query>();
    q->ticket = s->next_ticket++;
    q->graph_id = graph_id;
    q->root = root;
    q->dist_out = dist_out;
    q->int8 = (flags & BFS_DIST_INT8) != 0;
    q->submit_ns = now_ns();
    s->tickets[q->ticket] = q;
    s->pending[2 * (size_t)graph_id + (q->int8 ? 1 : 0)].push_back(q);
    s->stats.submitted += 1;
    *ticket = q->ticket;
    s->cv_work.notify_one();
    return BFS_OK;
}

bfs_status bfs_submit(bfs_server* s, int32_t graph_id, int32_t root, int32_t* dist_out,
                      bfs_ticket* ticket) {
    return bfs_submit_rows(s, graph_id, root, dist_out, 0, ticket);
}

bfs_status bfs_poll(bfs_server* s, bfs_ticket ticket) {
    if (!s) {
        set_error("null server");
        return BFS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_error("unknown ticket");
        return BFS_ERR_NOT_FOUND;
    }
    return it->second->status;
}

bfs_status bfs_wait(bfs_server* s, bfs_ticket ticket, int64_t timeout_us) {
    if (!s) {
        set_error("null server");
        return BFS_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_error("unknown ticket");
        return BFS_ERR_NOT_FOUND;
    }
    std::shared_ptr<Query> q = it->second;
    auto ready = [&] { return q->status != BFS_PENDING; };
    if (timeout_us < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    return q->status;
}

bfs_status bfs_ticket_times(bfs_server* s, bfs_ticket ticket, int64_t* submit_ns,
                            int64_t* launch_ns, int64_t* done_ns) {
    if (!s) {
        set_error("null server");
        return BFS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_error("unknown ticket");
        return BFS_ERR_NOT_FOUND;
    }
    const Query& q = *it->second;
    if (submit_ns) *submit_ns = q.submit_ns;
    if (launch_ns) *launch_ns = q.launch_ns;
    if (done_ns) *done_ns = q.done_ns;
    return q.status;
}

bfs_status bfs_release(bfs_server* s, bfs_ticket ticket) {
    if (!s) {
        set_error("null server");
        return BFS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_error("unknown ticket");
        return BFS_ERR_NOT_FOUND;
    }
    if (it->second->status == BFS_PENDING) {
        set_error("ticket still pending");
        return BFS_PENDING;
    }
    s->tickets.erase(it);
    return BFS_OK;
}

bfs_status bfs_server_replay_rows(bfs_server* s, int64_t nq, const int32_t* graph_ids,
                                  const int32_t* roots, const int64_t* arrival_ns,
                                  void* const* graph_bufs, const int32_t* bufs_per_graph,
                                  uint32_t flags, int64_t timeout_us, int64_t* done_ns,
                                  int32_t* status_out, int32_t* slot_out) {
    if (!s || nq < 0 || (nq > 0 && (!graph_ids || !roots || !arrival_ns || !graph_bufs ||
                                    !bufs_per_graph || !done_ns || !status_out))) {
        set_error("null argument");
        return BFS_ERR_INVALID_ARG;
    }
    if (flags & ~BFS_DIST_INT8) {
        set_error("unknown flag");
        return BFS_ERR_INVALID_ARG;
    }
    const size_t elt = (flags & BFS_DIST_INT8) ? 1 : 4;
    std::vector<int64_t> ns;  // vertices per graph
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto* g : s->graphs) ns.push_back(g->n);
    }
    const int ng = (int)ns.size();
    for (int64_t i = 0; i < nq; ++i)
        if (graph_ids[i] < 0 || graph_ids[i] >= ng || bufs_per_graph[graph_ids[i]] < 1 ||
            !graph_bufs[graph_ids[i]]) {
            set_error("replay: unknown graph or no buffers for it");
            return BFS_ERR_INVALID_ARG;
        }
    // per-graph free buffers and query lists (arrival order within a graph)
    std::vector<std::vector<int>> free_slots(ng);
    std::vector<std::vector<int64_t>> of_graph(ng);
    for (int g = 0; g < ng; ++g)
        for (int k = std::max(0, bufs_per_graph[g]) - 1; k >= 0; --k) free_slots[g].push_back(k);
    for (int64_t i = 0; i < nq; ++i) of_graph[graph_ids[i]].push_back(i);
    std::vector<bfs_ticket> tickets((size_t)nq, 0);
    std::vector<int> slot_of((size_t)nq, 0);
    std::vector<int64_t> fresh;  // submitted, not yet seen by the collector
    std::mutex mu;
    std::condition_variable cv;
    int64_t submitted = 0;
    int submitters_left = 0;
    bfs_status first_err = BFS_OK;
    for (int64_t i = 0; i < nq; ++i) {
        done_ns[i] = 0;
        status_out[i] = BFS_PENDING;
    }
    // collector: takes each query's result as soon as it completes (in any
    // order, so a long query does not hold the buffers of later ones)
    std::thread collector([&] {
        std::vector<int64_t> open, fin;
        std::vector<int64_t> opened_at;
        for (;;) {
            bool all_in = false;
            {
                std::lock_guard<std::mutex> lk(mu);
                for (int64_t j : fresh) {
                    open.push_back(j);
                    opened_at.push_back(now_ns());
                }
                fresh.clear();
                all_in = submitters_left == 0;
                if (open.empty() && all_in) break;
            }
            fin.clear();
            {
                std::unique_lock<std::mutex> lk(s->mu);
                auto any_done = [&] {
                    for (int64_t j : open) {
                        auto it = s->tickets.find(tickets[(size_t)j]);
                        if (it == s->tickets.end() || it->second->status != BFS_PENDING) return true;
                    }
                    return false;
                };
                s->cv_done.wait_for(lk, std::chrono::microseconds(200), any_done);
                for (size_t a = 0; a < open.size();) {
                    const int64_t j = open[a];
                    auto it = s->tickets.find(tickets[(size_t)j]);
                    const bool done = it == s->tickets.end() || it->second->status != BFS_PENDING;
                    const bool expired =
                        !done && timeout_us >= 0 && now_ns() - opened_at[a] > timeout_us * 1000;
                    if (!done && !expired) {
                        ++a;
                        continue;
                    }
                    if (it != s->tickets.end()) {
                        done_ns[j] = it->second->done_ns;
                        status_out[j] = expired ? BFS_ERR_TIMEOUT : it->second->status;
                        if (!expired) s->tickets.erase(it);
                    } else {
                        status_out[j] = BFS_ERR_NOT_FOUND;
                    }
                    fin.push_back(j);
                    open[a] = open.back();
                    open.pop_back();
                    opened_at[a] = opened_at.back();
                    opened_at.pop_back();
                }
            }
            if (!fin.empty()) {
                std::lock_guard<std::mutex> lk(mu);
                for (int64_t j : fin) {
                    if (slot_out) slot_out[j] = slot_of[(size_t)j];
                    if (status_out[j] == BFS_ERR_TIMEOUT) first_err = BFS_ERR_TIMEOUT;
                    else free_slots[graph_ids[j]].push_back(slot_of[(size_t)j]);
                }
                cv.notify_all();
            }
        }
    });
    // one submitter per graph: a graph whose buffers are all in use delays
    // only its own later queries, as independent clients would
    auto submit_graph = [&](int g) {
        for (int64_t i : of_graph[g]) {
            int slot = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (first_err != BFS_OK) break;
                auto any_free = [&] { return !free_slots[g].empty() || first_err != BFS_OK; };
                if (timeout_us < 0) cv.wait(lk, any_free);
                else if (!cv.wait_for(lk, std::chrono::microseconds(timeout_us), any_free)) {
                    first_err = BFS_ERR_TIMEOUT;
                    cv.notify_all();
                    break;
                }
                if (first_err != BFS_OK) break;
                slot = free_slots[g].back();
                free_slots[g].pop_back();
            }
            for (;;) {  // until the arrival time
                const int64_t now = now_ns();
                if (now >= arrival_ns[i]) break;
                if (arrival_ns[i] - now > 200000)
                    std::this_thread::sleep_for(std::chrono::nanoseconds(arrival_ns[i] - now - 100000));
            }
            bfs_ticket t = 0;
            char* row = static_cast<char*>(graph_bufs[g]) + (size_t)slot * (size_t)ns[(size_t)g] * elt;
            const bfs_status st = bfs_submit_rows(s, g, roots[i], row, flags, &t);
            std::lock_guard<std::mutex> lk(mu);
            if (st != BFS_OK) {
                first_err = st;
                free_slots[g].push_back(slot);
                cv.notify_all();
                break;
            }
            tickets[(size_t)i] = t;
            slot_of[(size_t)i] = slot;
            ++submitted;
            fresh.push_back(i);
            cv.notify_all();
        }
        std::lock_guard<std::mutex> lk(mu);
        --submitters_left;
        cv.notify_all();
    };
    std::vector<std::thread> submitters;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (int g = 0; g < ng; ++g)
            if (!of_graph[g].empty()) ++submitters_left;
    }
    for (int g = 0; g < ng; ++g)
        if (!of_graph[g].empty()) submitters.emplace_back(submit_graph, g);
    for (auto& th : submitters) th.join();
    collector.join();
    if (first_err != BFS_OK) return first_err;
    return BFS_OK;
}

bfs_status bfs_server_replay(bfs_server* s, int64_t nq, const int32_t* graph_ids,
                             const int32_t* roots, const int64_t* arrival_ns,
                             int32_t* const* graph_bufs, const int32_t* bufs_per_graph,
                             int64_t timeout_us, int64_t* done_ns, int32_t* status_out,
                             int32_t* slot_out) {
    return bfs_server_replay_rows(s, nq, graph_ids, roots, arrival_ns,
                                  reinterpret_cast<void* const*>(graph_bufs), bufs_per_graph, 0,
                                  timeout_us, done_ns, status_out, slot_out);
}

bfs_status bfs_replay_single(bfs_graph* const* graphs, int32_t ngraphs, int64_t nq,
                             const int32_t* graph_ids, const int32_t* roots,
                             const int64_t* arrival_ns, void* const* graph_bufs,
                             const int32_t* bufs_per_graph, uint32_t flags, void* stream,
                             int64_t* done_ns, int32_t* status_out) {
    if (!graphs || ngraphs < 1 || nq < 0 ||
        (nq > 0 && (!graph_ids || !roots || !arrival_ns || !graph_bufs || !bufs_per_graph ||
                    !done_ns || !status_out))) {
        set_error("null argument");
        return BFS_ERR_INVALID_ARG;
    }
    if (flags & ~BFS_DIST_INT8) {
        set_error("unknown flag");
        return BFS_ERR_INVALID_ARG;
    }
    const size_t elt = (flags & BFS_DIST_INT8) ? 1 : 4;
    for (int64_t i = 0; i < nq; ++i) {
        const int g = graph_ids[i];
        if (g < 0 || g >= ngraphs || !graphs[g] || bufs_per_graph[g] < 1 || !graph_bufs[g]) {
            set_error("replay: unknown graph or no buffers for it");
            return BFS_ERR_INVALID_ARG;
        }
    }
    std::vector<int64_t> used((size_t)ngraphs, 0);
    bfs_status first_err = BFS_OK;
    for (int64_t i = 0; i < nq; ++i) {
        const int g = graph_ids[i];
        for (;;) {  // until the arrival time (queries run in arrival order)
            const int64_t now = now_ns();
            if (now >= arrival_ns[i]) break;
            if (arrival_ns[i] - now > 200000)
                std::this_thread::sleep_for(std::chrono::nanoseconds(arrival_ns[i] - now - 100000));
        }
        char* out = static_cast<char*>(graph_bufs[g]) +
                    (size_t)(used[(size_t)g]++ % bufs_per_graph[g]) * (size_t)graphs[g]->n * elt;
        const bfs_status st = bfs_run(graphs[g], roots[i], reinterpret_cast<int32_t*>(out), nullptr,
                                      stream, BFS_OUT_HOST | (flags & BFS_DIST_INT8));
        done_ns[i] = now_ns();
        status_out[i] = st;
        if (st != BFS_OK && first_err == BFS_OK) first_err = st;
    }
    return first_err;
}

bfs_status bfs_server_get_stats(bfs_server* s, bfs_server_stats* out) {
    if (!s || !out) {
        set_error("null argument");
        return BFS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return BFS_OK;
}

bfs_status bfs_server_destroy(bfs_server* s) {
    if (!s) {
        set_error("null server");
        return BFS_ERR_INVALID_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& q : s->pending) {
            for (auto& x : q) x->status = BFS_ERR_CANCELLED;
            q.clear();
        }
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    if (s->dispatcher.joinable()) s->dispatcher.join();
    cudaSetDevice(s->ctx->device);
    for (auto& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.event);
        cudaEventDestroy(sl.kevent);
    }
    delete s->mem;
    s->ctx->mem->release(s->arena);
    delete s;
    return BFS_OK;
}

}  // extern "C"
