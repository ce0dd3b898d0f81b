// bfs_paths.cu -- shortest-path counts and weight-filtered traversal on a
// CSR the caller holds on the device (bfs_run_paths).
//
// Section "Top Down Vs. Bottom Up" names two uses of BFS that a bottom-up
// level cannot serve: betweenness-type computations, which need every
// shortest path, and weight-filtering BFS, which follows only the edges of
// given weights.  Both examine every entry leaving the frontier, so this
// path is top-down only.  It computes, for the subgraph of entries e with
// lo <= weight[e] <= hi, hops[v] (the BFS distance, -1 unreached) and
// sigma[v] (the number of shortest root -> v paths) -- the forward phase of
// Brandes' betweenness algorithm in its level-synchronous form.
//
// Per level:
//   1. the out-degree of every frontier vertex (rows checked against nnz);
//   2. an exclusive scan of those degrees (the frontier's entries laid end
//      to end);
//   3. an edge-balanced expansion: CTAs take tiles of 2048 consecutive
//      frontier entries, each thread finds its entry's vertex by binary
//      search in the tile's span of the scan, so a hub's row spreads over
//      many CTAs, light rows share one, and consecutive threads read
//      consecutive columns.  A kept entry v -> u whose target has no
//      distance, or already has level + 1, lies on a shortest path: it sets
//      hops[u] = level + 1 and adds sigma[v] to sigma[u] by a
//      double-precision atomic add.  sigma[v] is final when level L is
//      expanded: every predecessor sits at level L - 1;
//   4. the next frontier collected from the distances (hops = level + 1).
// The host reads the next frontier size after each level.  Every column
// index is checked against n and every row against nnz before use: a bad
// CSR ends the call with BFS_ERR_INVALID_GRAPH, never an out-of-range
// access.
#include <cuda_runtime.h>

#include <algorithm>

#include "bfs_runtime.h"

namespace bfs {

cudaError_t exclusive_scan_i64(const int64_t* in, long long n, int64_t* out, int64_t* tmp,
                               cudaStream_t s);

namespace {

constexpr int kPathThreads = 256;
constexpr int kPathPerThread = 8;
constexpr long long kPathTile = (long long)kPathThreads * kPathPerThread;  // entries per tile

struct PathCtl {
    unsigned long long tail;   // entries written to the next frontier
    unsigned long long edges;  // entries of the expanded rows so far
    int bad;                   // a row or column index out of range was met
    int pad[3];
};

__global__ void paths_init(int32_t* hops, double* sigma, long long n, int32_t root, int32_t* fr,
                           PathCtl* ctl) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        hops[i] = i == root ? 0 : -1;
        sigma[i] = i == root ? 1.0 : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        fr[0] = root;
        ctl->tail = 0;
        ctl->edges = 0;
        ctl->bad = 0;
    }
}

// deg[i] = out-degree of frontier vertex fr[i]; a row outside [0, nnz]
// counts as empty and raises the error flag.
__global__ void paths_degrees(const int64_t* off, long long nnz, const int32_t* fr, long long nfr,
                              int64_t* deg, PathCtl* ctl) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nfr; i += stride) {
        const int32_t v = fr[i];
        const long long b = off[v], e = off[v + 1];
        long long d = e - b;
        if (b < 0 || d < 0 || e > nnz) {
            ctl->bad = 1;
            d = 0;
        }
        deg[i] = d;
    }
}

// Largest i in [a, b] with prefix[i] <= key (prefix[a] <= key required).
__device__ __forceinline__ long long owner_of(const int64_t* prefix, long long a, long long b,
                                             long long key) {
    while (a < b) {
        const long long m = (a + b + 1) >> 1;
        if (prefix[m] <= key) a = m;
        else b = m - 1;
    }
    return a;
}

// Level L's expansion.  A kept entry v -> u is a shortest-path edge exactly
// when u has no distance yet or already has L + 1: the entry itself puts u
// at L + 1.  So each such entry stores hops[u] = L + 1 (every writer stores
// the same value) and adds sigma[v] to sigma[u] with an atomic whose result
// is not used -- no compare-and-swap, no queue reservation, nothing a thread
// waits for; the next frontier is collected afterwards (paths_collect).
// Each thread takes 8 entries of the tile and issues their distance loads
// together before the first update.
__global__ void __launch_bounds__(kPathThreads)
paths_expand(const int64_t* off, const int32_t* col, const int32_t* weight, int32_t lo, int32_t hi,
             long long n, const int32_t* fr, long long nfr, const int64_t* prefix, int level,
             int32_t* hops, double* sigma, PathCtl* ctl) {
    __shared__ long long s_span[2];
    const long long total = prefix[nfr];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->edges += (unsigned long long)total;
    const int32_t nxt_level = level + 1;
    for (long long t0 = (long long)blockIdx.x * kPathTile; t0 < total;
         t0 += (long long)gridDim.x * kPathTile) {
        const long long t1 = t0 + kPathTile < total ? t0 + kPathTile : total;
        // the frontier entries whose rows this tile covers: [s_span[0], s_span[1]]
        if (threadIdx.x < 2)
            s_span[threadIdx.x] = owner_of(prefix, 0, nfr - 1, threadIdx.x == 0 ? t0 : t1 - 1);
        __syncthreads();
        const long long first = s_span[0], last = s_span[1];
        int32_t u[kPathPerThread];
        double sv[kPathPerThread];
        bool take[kPathPerThread];
#pragma unroll
        for (int j = 0; j < kPathPerThread; ++j) {
            const long long e = t0 + (long long)j * kPathThreads + threadIdx.x;
            take[j] = false;
            u[j] = 0;
            sv[j] = 0.0;
            if (e < t1) {
                const long long i = owner_of(prefix, first, last, e);
                const int32_t v = fr[i];
                const long long k = off[v] + (e - prefix[i]);
                u[j] = col[k];
                take[j] = weight == nullptr || (weight[k] >= lo && weight[k] <= hi);
                if (take[j] && (u[j] < 0 || (long long)u[j] >= n)) {
                    ctl->bad = 1;
                    take[j] = false;
                }
                if (take[j]) sv[j] = sigma[v];
            }
        }
        int32_t h[kPathPerThread];
#pragma unroll
        for (int j = 0; j < kPathPerThread; ++j) h[j] = take[j] ? hops[u[j]] : 0;
#pragma unroll
        for (int j = 0; j < kPathPerThread; ++j) {
            if (take[j] && (h[j] == -1 || h[j] == nxt_level)) {
                if (h[j] == -1) hops[u[j]] = nxt_level;
                atomicAdd(sigma + u[j], sv[j]);
            }
        }
        __syncthreads();
    }
}

// The next frontier: every vertex whose distance is `level`, in vertex order
// within each warp (one queue reservation per warp).
__global__ void paths_collect(const int32_t* hops, long long n, int32_t level, int32_t* next,
                              PathCtl* ctl) {
    const unsigned lane = threadIdx.x & 31u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nround = (n + 31) / 32 * 32;  // warp-uniform trip count
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nround; v += stride) {
        const bool in = v < n && hops[v] == level;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (m == 0u) continue;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if ((int)lane == leader) base = atomicAdd(&ctl->tail, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        const unsigned long long slot = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
        if (in) {
            if (slot < (unsigned long long)n) next[slot] = (int32_t)v;
            else ctl->bad = 1;
        }
    }
}

// Device memory of `device` (or managed memory): host and other GPUs'
// pointers are refused before any kernel could touch them.
bool on_device(const void* p, int device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == device) ||
           a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace bfs

using namespace bfs;

extern "C" bfs_status bfs_run_paths(bfs_context* ctx, const int64_t* row_off, const int32_t* col,
                                    const int32_t* weight, int64_t n, int64_t nnz, int32_t w_lo,
                                    int32_t w_hi, int32_t root, int32_t* hops, double* sigma,
                                    void* stream, bfs_paths_stats* stats) {
    if (!ctx || !row_off || !hops || !sigma || (nnz > 0 && !col)) {
        set_error("paths: null context, offsets, column array or output");
        return BFS_ERR_INVALID_ARG;
    }
    if (n < 1 || n > (int64_t)INT32_MAX || nnz < 0) {
        set_error("paths: n must lie in [1, 2^31 - 1] and nnz must not be negative");
        return BFS_ERR_INVALID_ARG;
    }
    if (root < 0 || root >= n) {
        set_error("paths: root out of range");
        return BFS_ERR_ROOT_RANGE;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const int dv = ctx->device;
    if (!on_device(row_off, dv) || (nnz > 0 && !on_device(col, dv)) ||
        (weight && !on_device(weight, dv)) || !on_device(hops, dv) || !on_device(sigma, dv)) {
        set_error("paths: every array must be device memory of the context's GPU");
        return BFS_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceAllocator* m = ctx->mem;
    const size_t nz = (size_t)n;
    int32_t* fr[2] = {static_cast<int32_t*>(m->alloc(nz * 4 + 64)),
                      static_cast<int32_t*>(m->alloc(nz * 4 + 64))};
    int64_t* deg = static_cast<int64_t*>(m->alloc(nz * 8 + 64));
    int64_t* prefix = static_cast<int64_t*>(m->alloc(nz * 8 + 64));
    int64_t* tmp = static_cast<int64_t*>(m->alloc((nz / 256 + 4) * 8));
    PathCtl* ctl = static_cast<PathCtl*>(m->alloc(sizeof(PathCtl)));
    auto release = [&]() {
        m->release(fr[0]);
        m->release(fr[1]);
        m->release(deg);
        m->release(prefix);
        m->release(tmp);
        m->release(ctl);
    };
    if (!fr[0] || !fr[1] || !deg || !prefix || !tmp || !ctl) {
        release();
        set_error("paths: device memory exhausted");
        return BFS_ERR_NO_MEMORY;
    }
    const int sms = ctx->sms;
    paths_init<<<sms * 4, 256, 0, s>>>(hops, sigma, n, root, fr[0], ctl);
    bfs_paths_stats st{};
    long long nfr = 1, reached = 1;
    int cur = 0;
    for (int level = 0; nfr > 0 && e == cudaSuccess; ++level) {
        st.levels = level + 1;
        const int gd = (int)std::min<long long>((long long)sms * 8, (nfr + 255) / 256);
        paths_degrees<<<gd, 256, 0, s>>>(row_off, nnz, fr[cur], nfr, deg, ctl);
        e = exclusive_scan_i64(deg, nfr, prefix, tmp, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->tail, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) break;
        paths_expand<<<sms * 8, kPathThreads, 0, s>>>(row_off, col, weight, w_lo, w_hi, n, fr[cur],
                                                      nfr, prefix, level, hops, sigma, ctl);
        paths_collect<<<sms * 8, 256, 0, s>>>(hops, n, level + 1, fr[cur ^ 1], ctl);
        e = cudaGetLastError();
        unsigned long long h_tail = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_tail, &ctl->tail, sizeof(h_tail), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        nfr = (long long)std::min<unsigned long long>(h_tail, (unsigned long long)n);
        reached += nfr;
        cur ^= 1;
    }
    PathCtl h_ctl{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_ctl, ctl, sizeof(h_ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "paths traversal");
    if (h_ctl.bad) {
        set_error("paths: a row offset or column index lies outside the CSR");
        return BFS_ERR_INVALID_GRAPH;
    }
    st.reached = reached;
    st.edges_scanned = (int64_t)h_ctl.edges;
    if (stats) *stats = st;
    return BFS_OK;
}
