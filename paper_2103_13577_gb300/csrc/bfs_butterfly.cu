// bfs_butterfly.cu -- ButterFly BFS (Algorithm 2) emulated on one GPU.
//
// P virtual compute nodes share the device.  Every node keeps its own
// distance array d_local[g] (Algorithm 2 initialisation), owns one 1D vertex
// range of about M/P adjacency entries (Section "Graph Partitioning": vertex
// ids consecutive, near-equal edge counts) and two queues: Q_local (owned
// frontier) and Q_global (every vertex the node found at this level).
//
// Phase 1 (traversal): node g expands only its Q_local; an unvisited
// neighbour u (d_local[g][u] = infinity) is claimed with an atomic
// compare-and-swap, whose success gates d_local[g][u] = level + 1 and the
// enqueue into Q_global[g] (and Q_local[g] when g owns u).
//
// Phase 2 (butterfly synchronisation, Section "Synchronizing with
// ButterFlies" and "Fanout & Trade-offs"): log_r(P) rounds with radix r =
// max(2, fanout).  In round i node g receives the Q_global of every node
// whose base-r id differs from g only in digit i (fanout 1: g XOR 2^i, the
// recursive doubling of the fanout-one figure), as it stood when the round
// began, filters it by its own d_local, and enqueues the new vertices as in
// Phase 1.  After the last round every node knows the whole next frontier.
//
// This is an emulation for correctness and accounting (messages, entries
// moved, buffer sizes): nodes run one after another on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "bfs_runtime.h"

namespace bfs {
namespace {

__device__ __forceinline__ void append2(bool win, bool own, int32_t u, int32_t* qg,
                                        unsigned long long* qg_cnt, int32_t* ql,
                                        unsigned long long* ql_cnt) {
    const unsigned lane = threadIdx.x & 31;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const unsigned mg = __ballot_sync(0xffffffffu, win);
    if (mg) {
        unsigned long long base = 0;
        const int leader = __ffs(mg) - 1;
        if ((int)lane == leader) base = atomicAdd(qg_cnt, (unsigned long long)__popc(mg));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (win) qg[base + __popc(mg & lt)] = u;
    }
    const unsigned ml = __ballot_sync(0xffffffffu, win && own);
    if (ml) {
        unsigned long long base = 0;
        const int leader = __ffs(ml) - 1;
        if ((int)lane == leader) base = atomicAdd(ql_cnt, (unsigned long long)__popc(ml));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (win && own) ql[base + __popc(ml & lt)] = u;
    }
}

// Phase 1 for one node: one warp per frontier vertex.
__global__ void bf_expand(const int64_t* off, const int32_t* col, int32_t* dl, const int32_t* fr,
                          long long nfr, int32_t* qg, unsigned long long* qg_cnt, int32_t* qln,
                          unsigned long long* qln_cnt, long long own_lo, long long own_hi,
                          int level) {
    const long long nwarps = (long long)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    for (long long i = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < nfr;
         i += nwarps) {
        const int32_t v = fr[i];
        const long long b = off[v], e = off[v + 1];
        for (long long k0 = b; k0 < e; k0 += 32) {
            const long long k = k0 + lane;
            bool win = false;
            int32_t u = 0;
            if (k < e) {
                u = col[k];
                if (dl[u] == -1) win = atomicCAS(dl + u, -1, level + 1) == -1;
            }
            append2(win, u >= own_lo && u < own_hi, u, qg, qg_cnt, qln, qln_cnt);
        }
    }
}

// Phase 2 for one (receiver, sender) pair: the sender's Q_global prefix of
// `cnt` entries, filtered by the receiver's d_local.
__global__ void bf_receive(int32_t* dl, const int32_t* qsrc, long long cnt, int32_t* qg,
                           unsigned long long* qg_cnt, int32_t* qln, unsigned long long* qln_cnt,
                           long long own_lo, long long own_hi, int level) {
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long rounds = (cnt + 31) / 32 * 32;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < rounds; i += nthreads) {
        bool win = false;
        int32_t v = 0;
        if (i < cnt) {
            v = qsrc[i];
            if (dl[v] == -1) win = atomicCAS(dl + v, -1, level + 1) == -1;
        }
        append2(win, v >= own_lo && v < own_hi, v, qg, qg_cnt, qln, qln_cnt);
    }
}

__global__ void bf_fill(int32_t* p, long long n, int32_t value) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = value;
}

// Seeds the root in every node (d_local[g][root] = 0), its owner's Q_local.
__global__ void bf_seed(int32_t* dl_all, long long n, int nodes, int32_t root, int32_t* ql_owner,
                        unsigned long long* ql_cnt_owner) {
    for (int g = threadIdx.x; g < nodes; g += blockDim.x) dl_all[(long long)g * n + root] = 0;
    if (threadIdx.x == 0) {
        ql_owner[0] = root;
        *ql_cnt_owner = 1;
    }
}

// dist (caller numbering) from node 0, and the number of vertices on which
// any node disagrees with node 0.
__global__ void bf_output(const int32_t* dl_all, long long n, int nodes, const int32_t* new2old,
                          int32_t* dist, unsigned long long* disagree) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long bad = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t d0 = dl_all[v];
        for (int g = 1; g < nodes; ++g) bad += dl_all[(long long)g * n + v] != d0;
        dist[new2old ? new2old[v] : v] = d0;
    }
    if (bad) atomicAdd(disagree, bad);
}

}  // namespace
}  // namespace bfs

using namespace bfs;

extern "C" bfs_status bfs_butterfly_schedule(int32_t nodes, int32_t fanout, int32_t round,
                                             int32_t node, int32_t* partners, int32_t* count) {
    if (!partners || !count || nodes < 1 || nodes > 256 || fanout < 1 || fanout > 16 || round < 0 ||
        node < 0 || node >= nodes) {
        set_error("butterfly schedule: bad argument");
        return BFS_ERR_INVALID_ARG;
    }
    const int radix = std::max(2, (int)fanout);
    long long stride = 1;
    for (int i = 0; i < round; ++i) stride *= radix;
    if (stride >= nodes) {
        set_error("butterfly schedule: round beyond the last");
        return BFS_ERR_INVALID_ARG;
    }
    const long long digit = (node / stride) % radix;
    const long long base = node - digit * stride;
    int c = 0;
    for (int d = 0; d < radix; ++d) {
        const long long p = base + d * stride;
        if (p != node && p < nodes) partners[c++] = (int32_t)p;
    }
    *count = c;
    return BFS_OK;
}

extern "C" bfs_status bfs_run_butterfly(bfs_graph* g, int32_t root, int32_t nodes, int32_t fanout,
                                        int32_t* dist, void* stream, bfs_butterfly_stats* stats) {
    TraceRange tr("bfs_run_butterfly", root);
    if (!g || !dist) {
        set_error("butterfly: null graph or dist");
        return BFS_ERR_INVALID_ARG;
    }
    if (root < 0 || root >= g->n) {
        set_error("butterfly: root out of range");
        return BFS_ERR_ROOT_RANGE;
    }
    const int radix = std::max(2, (int)fanout);
    if (nodes < 1 || nodes > 256 || fanout < 1 || fanout > 16) {
        set_error("butterfly: nodes must be 1..256 and fanout 1..16");
        return BFS_ERR_INVALID_ARG;
    }
    int rounds = 0;
    for (long long p = 1; p < nodes; p *= radix) ++rounds;
    long long pw = 1;
    for (int i = 0; i < rounds; ++i) pw *= radix;
    if (pw != nodes) {
        set_error("butterfly: nodes must be a power of max(2, fanout)");
        return BFS_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(g->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = g->n;
    const int sms = g->ctx->sms;

    // 1D partition: node k owns [lo[k], lo[k+1]) with about k*nnz/P entries before it
    std::vector<long long> lo(nodes + 1, 0);
    {
        std::vector<int64_t> h_off(n + 1);
        e = cudaMemcpy(h_off.data(), g->d_off, (n + 1) * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "butterfly partition");
        for (int k = 1; k < nodes; ++k) {
            const long long target = (long long)((double)g->nnz * k / nodes);
            lo[k] = std::lower_bound(h_off.begin(), h_off.end(), (int64_t)target) - h_off.begin();
            lo[k] = std::min(std::max(lo[k], lo[k - 1]), n);
        }
        lo[nodes] = n;
    }
    DeviceAllocator* m = g->ctx->mem;
    int32_t* dl = static_cast<int32_t*>(m->alloc((size_t)nodes * n * 4));
    int32_t* qg = static_cast<int32_t*>(m->alloc((size_t)nodes * n * 4));
    int32_t* ql[2] = {static_cast<int32_t*>(m->alloc((size_t)n * 4 + 64)),
                      static_cast<int32_t*>(m->alloc((size_t)n * 4 + 64))};
    unsigned long long* cnt = static_cast<unsigned long long*>(m->alloc((size_t)(3 * nodes + 1) * 8));
    auto release = [&]() {
        m->release(dl);
        m->release(qg);
        m->release(ql[0]);
        m->release(ql[1]);
        m->release(cnt);
    };
    if (!dl || !qg || !ql[0] || !ql[1] || !cnt) {
        release();
        set_error("butterfly: device memory exhausted");
        return BFS_ERR_NO_MEMORY;
    }
    unsigned long long* qg_cnt = cnt;                // [nodes]
    unsigned long long* ql_cnt[2] = {cnt + nodes, cnt + 2 * nodes};
    unsigned long long* disagree = cnt + 3 * nodes;
    int32_t dev_root = root;
    if (g->relabelled) {
        e = cudaMemcpy(&dev_root, g->d_old2new + root, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(e, "butterfly root");
        }
    }
    int owner = 0;
    while (owner + 1 < nodes && dev_root >= lo[owner + 1]) ++owner;

    bf_fill<<<sms * 4, 256, 0, s>>>(dl, (long long)nodes * n, -1);
    e = cudaMemsetAsync(cnt, 0, (size_t)(3 * nodes + 1) * 8, s);
    bf_seed<<<1, 256, 0, s>>>(dl, n, nodes, dev_root, ql[0] + lo[owner], ql_cnt[0] + owner);

    bfs_butterfly_stats st{};
    st.nodes = nodes;
    st.radix = radix;
    st.rounds_per_level = rounds;
    std::vector<unsigned long long> h_ql(nodes), h_qg(nodes);
    int cur = 0;
    for (int level = 0; e == cudaSuccess; ++level) {
        TraceRange lv("level", level);
        e = cudaMemcpyAsync(h_ql.data(), ql_cnt[cur], nodes * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        unsigned long long total = 0;
        for (int k = 0; k < nodes; ++k) total += h_ql[k];
        if (total == 0) break;
        st.levels = level + 1;
        const int nxt = cur ^ 1;
        e = cudaMemsetAsync(qg_cnt, 0, nodes * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ql_cnt[nxt], 0, nodes * 8, s);
        // Phase 1: every node expands its owned frontier
        for (int k = 0; k < nodes && e == cudaSuccess; ++k) {
            if (h_ql[k] == 0) continue;
            bf_expand<<<sms * 4, 256, 0, s>>>(g->d_off, g->d_col, dl + (long long)k * n,
                                                ql[cur] + lo[k], (long long)h_ql[k],
                                                qg + (long long)k * n, qg_cnt + k,
                                                ql[nxt] + lo[k], ql_cnt[nxt] + k, lo[k], lo[k + 1],
                                                level);
        }
        // Phase 2: butterfly rounds over the base-r digits of the node ids
        long long stride = 1;
        for (int i = 0; i < rounds && e == cudaSuccess; ++i, stride *= radix) {
            e = cudaMemcpyAsync(h_qg.data(), qg_cnt, nodes * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            for (int k = 0; k < nodes; ++k) st.max_global_queue = std::max<long long>(st.max_global_queue, (long long)h_qg[k]);
            std::vector<unsigned long long> snap = h_qg;
            for (int k = 0; k < nodes && e == cudaSuccess; ++k) {
                int32_t partners[16], np = 0;
                bfs_butterfly_schedule(nodes, fanout, i, k, partners, &np);
                long long buffer = 0;
                for (int pi = 0; pi < np; ++pi) {
                    const int p = partners[pi];
                    st.messages += 1;
                    st.message_entries += (long long)snap[p];
                    buffer += (long long)snap[p];
                    if (snap[p] == 0) continue;
                    const int blocks = (int)std::min<long long>(sms * 4, ((long long)snap[p] + 255) / 256);
                    bf_receive<<<blocks, 256, 0, s>>>(dl + (long long)k * n, qg + (long long)p * n,
                                                      (long long)snap[p], qg + (long long)k * n,
                                                      qg_cnt + k, ql[nxt] + lo[k], ql_cnt[nxt] + k,
                                                      lo[k], lo[k + 1], level);
                }
                st.max_round_buffer_entries = std::max<long long>(st.max_round_buffer_entries, buffer);
            }
        }
        cur = nxt;
    }
    unsigned long long h_dis = 0;
    if (e == cudaSuccess) {
        bf_output<<<sms * 4, 256, 0, s>>>(dl, n, nodes, g->relabelled ? g->d_new2old : nullptr, dist,
                                          disagree);
        e = cudaMemcpyAsync(&h_dis, disagree, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    release();
    if (e != cudaSuccess) return cuda_fail(e, "butterfly traversal");
    st.node_disagreements = (long long)h_dis;
    if (stats) *stats = st;
    return BFS_OK;
}
