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
// One cooperative persistent launch runs the whole level loop; a grid
// barrier (bounded by %globaltimer) separates its phases, so the host waits
// once per traversal, not once per level.  Per level L:
//   1. expansion: the frontier queue holds each vertex with the exclusive
//      prefix of the frontier's degrees (its first entry's position in the
//      level's entry sequence), so CTAs take tiles of 2048 consecutive
//      entries; a chunk-start table (written when the vertices are queued)
//      gives a tile's first and last queue entries, the span between them is
//      staged in shared memory and each thread finds its entries' rows by
//      binary search there, so a
//      hub's row spreads over many CTAs, light rows share one, and
//      consecutive threads read consecutive columns.  A kept entry v -> u
//      lies on a shortest path exactly when u was not reached at level <= L
//      (one bit of the visited bitmap, read without atomics: it does not
//      change during the phase): such an entry marks u in the next-frontier
//      bitmap and adds sigma[v] to sigma[u] (reductions whose results are not
//      used, so nothing waits for them).  sigma[v] is final when level L is
//      expanded: every predecessor sits at level L - 1;
//   2. collection: warps scan the next-frontier bitmap, give each marked
//      vertex hops = L + 1, fold the bitmap into the visited one and clear
//      it, and append the marked vertices with out-edges to the next queue
//      -- one packed 64-bit atomicAdd per warp round reserves queue slots
//      and the entry prefix together (count << 34 | entries) -- and mark in
//      the chunk-start table every tile whose first entry they hold.
// Every row is checked against [0, nnz] and every kept column index against
// [0, n) before use: a bad CSR ends the call with BFS_ERR_INVALID_GRAPH,
// never an out-of-range access.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "bfs_runtime.h"

namespace bfs {

namespace {

constexpr int kPathThreads = 256;
constexpr int kPathWarps = kPathThreads / 32;
constexpr int kPathPerLane = 8;
constexpr int kPathTile = 32 * kPathPerLane;                // entries per warp tile
constexpr int kPathMinBlocks = 3;
constexpr int kPackShift = 34;                              // count << 34 | entries
constexpr unsigned long long kPackMask = (1ull << kPackShift) - 1ull;

struct PathCtl {
    unsigned long long packed[2];   // queue of parity p: (entries << 34) | entry prefix
    unsigned long long edges;       // entries of the reached rows
    unsigned long long reached;     // vertices with hops >= 0
    unsigned long long arrived;     // barrier arrivals of the launch; bit 63: a CTA gave up
    unsigned int exit_count;
    int bad;                        // a row or column index out of range was met
    int status;                     // 1: a grid-barrier wait gave up
    int levels;                     // max hops + 1
    int pad;
};

struct PathParams {
    const int64_t* off;
    const int32_t* col;
    const int32_t* weight;          // nullable: every entry kept
    int32_t lo, hi;
    long long n, nnz;
    int32_t root;
    int32_t* hops;
    double* sigma;
    uint32_t* vis;                  // vertices reached at a level <= L
    uint32_t* mark;                 // vertices reached at level L + 1 (being built)
    int32_t* qv[2];                 // frontier vertices
    int64_t* qe[2];                 // their first entry's position in the level's sequence
    int64_t* qk[2];                 // row start minus that position: entry e of the sequence
                                    // is col[e + qk] for the vertex holding it
    int32_t* qc[2];                 // tile t's first queue entry: the one holding entry t * 256
    long long qc_cap;               // slots of each qc array
    PathCtl* ctl;
    long long timeout_ns;
};

__device__ __forceinline__ unsigned long long timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All CTAs are co-resident (cooperative launch).  Thread 0 of each CTA adds
// its arrival to a 64-bit word that only grows during the launch; the k-th
// barrier is complete once it reaches k * gridDim.x (`epoch`, thread 0's in
// shared memory, counts the barriers passed, the same in every CTA), so an arrival is one
// fire-and-forget reduction and the wait a loop of acquire loads.  A wait
// longer than timeout_ns records the failure and sets bit 63, which makes
// every CTA leave; the return value says whether to go on.
constexpr unsigned long long kPathGaveUp = 1ull << 63;

__device__ bool path_barrier(const PathParams& P, unsigned long long& epoch) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* const word = &P.ctl->arrived;
        const unsigned long long target = ++epoch * gridDim.x;
        int ok = 1;
        __threadfence();
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(word) : "memory");
        unsigned long long t0 = 0ull;
        for (;;) {
            unsigned long long a;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(a) : "l"(word) : "memory");
            if (a & kPathGaveUp) { ok = 0; break; }
            if (a >= target) break;
            const unsigned long long t = timer_ns();
            if (t0 == 0ull) {
                t0 = t;
            } else if (t - t0 > (unsigned long long)P.timeout_ns) {
                atomicExch(&P.ctl->status, 1);
                atomicOr(word, kPathGaveUp);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (unsigned)d) x += y;
    }
    return x;
}

// Records, for every tile whose first entry falls in [eo, eo + deg), that
// queue entry pos holds it (chunk-start table of the queue being built).
__device__ __forceinline__ void mark_tiles(const PathParams& P, int nxt, long long pos, long long eo,
                                           long long deg) {
    const long long c0 = (eo + kPathTile - 1) / kPathTile, c1 = (eo + deg - 1) / kPathTile;
    for (long long c = c0; c <= c1; ++c) {
        if (c < P.qc_cap) P.qc[nxt][c] = (int32_t)pos;
        else P.ctl->bad = 1;
    }
}

// Level L's expansion over the queue of parity cur (cnt vertices, E entries).
// Warps take tiles of 256 consecutive entries (round robin over the grid, no
// CTA barriers): lane 0 reads the tile's first and last queue entries from
// the chunk-start table, the warp stages that span (vertex, first entry
// relative to the tile, row shift) in its shared-memory slice, and each lane
// finds the row of its 8 entries (tile entries lane + 32 j) by a search that
// starts at its previous entry's row.  Everything written during the launch
// (queues, bitmaps, sigma) is read through L2 (ld.cg): an L1 or
// read-only-cache copy could predate the write.
__device__ void expand_paths(const PathParams& P, int cur, long long cnt, long long E) {
    __shared__ int32_t s_rel[kPathWarps][kPathTile + 1];   // first tile entry of each span entry
    __shared__ long long s_k[kPathWarps][kPathTile + 1];    // row shift
    __shared__ double s_sig[kPathWarps][kPathTile + 1];     // sigma of the row's vertex (final)
    const unsigned lane = threadIdx.x & 31u;
    const int w = threadIdx.x >> 5;
    int32_t* const rel = s_rel[w];
    long long* const ks = s_k[w];
    double* const sg = s_sig[w];
    const int32_t* qv = P.qv[cur];
    const int64_t* qe = P.qe[cur];
    const int64_t* qk = P.qk[cur];
    const int32_t* qc = P.qc[cur];
    const long long tiles = (E + kPathTile - 1) / kPathTile;
    const long long nwarps = (long long)gridDim.x * kPathWarps;
    for (long long t = (long long)blockIdx.x * kPathWarps + w; t < tiles; t += nwarps) {
        const long long t0 = t * kPathTile;
        const int len = (int)min((long long)kPathTile, E - t0);
        // the tile's entries: from the one holding its first entry to the one
        // holding the next tile's first entry (which may start exactly at the
        // tile's end and then contributes nothing)
        long long first = 0, last = 0;
        if (lane == 0) {
            first = min((long long)__ldcg(qc + t), cnt - 1);
            last = t + 1 < tiles ? min((long long)__ldcg(qc + t + 1), cnt - 1) : cnt - 1;
        }
        first = __shfl_sync(0xffffffffu, first, 0);
        last = __shfl_sync(0xffffffffu, last, 0);
        // every queued vertex has edges: at most kPathTile + 1 entries
        const int span = (int)max(0ll, min(last - first + 1, (long long)kPathTile + 1));
        for (int i = (int)lane; i < span; i += 32) {
            const long long eo = __ldcg(qe + first + i);
            rel[i] = (int32_t)max(eo - t0, 0ll);
            ks[i] = __ldcg(qk + first + i);
            sg[i] = __ldcg(P.sigma + __ldcg(qv + first + i));
        }
        __syncwarp();
        int32_t u[kPathPerLane];
        double sv[kPathPerLane];
        bool take[kPathPerLane];
        int o = 0;
#pragma unroll
        for (int j = 0; j < kPathPerLane; ++j) {
            const int r = j * 32 + (int)lane;   // tile entry
            take[j] = false;
            u[j] = 0;
            sv[j] = 0.0;
            if (r < len) {
                // rows are in order: search from the previous entry's row
                if (o + 1 < span && rel[o + 1] <= r) {
                    int a = o + 1, b = span - 1;
                    while (a < b) {
                        const int m = (a + b + 1) >> 1;
                        if (rel[m] <= r) a = m;
                        else b = m - 1;
                    }
                    o = a;
                }
                const long long k = t0 + r + ks[o];
                sv[j] = sg[o];
                u[j] = __ldcs(P.col + k);
                if (P.weight) {
                    const int32_t wt = __ldcs(P.weight + k);
                    take[j] = wt >= P.lo && wt <= P.hi;
                } else {
                    take[j] = true;
                }
            }
        }
        // visited probes: a plain (L1-cacheable) read first -- an L1 copy
        // from an earlier level can only show clear a bit that is set since,
        // never the reverse -- and a read through L2 for the bits it shows
        // clear, which decides
        uint32_t wd[kPathPerLane];
#pragma unroll
        for (int j = 0; j < kPathPerLane; ++j) {
            if (take[j] && (u[j] < 0 || (long long)u[j] >= P.n)) {
                P.ctl->bad = 1;
                take[j] = false;
            }
            wd[j] = take[j] ? P.vis[u[j] >> 5] : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < kPathPerLane; ++j)
            if (!((wd[j] >> (u[j] & 31)) & 1u)) wd[j] = __ldcg(P.vis + (u[j] >> 5));
#pragma unroll
        for (int j = 0; j < kPathPerLane; ++j) {
            if (take[j] && !((wd[j] >> (u[j] & 31)) & 1u)) {
                atomicOr(P.mark + (u[j] >> 5), 1u << (u[j] & 31));
                atomicAdd(P.sigma + u[j], sv[j]);
            }
        }
        __syncwarp();
    }
}

// Level L's collection into the queue of parity nxt.
__device__ void collect_paths(const PathParams& P, int level, int nxt) {
    const unsigned lane = threadIdx.x & 31u;
    const long long words = (P.n + 31) / 32;
    const long long groups = (words + 31) / 32;
    const long long nwarps = (long long)gridDim.x * (kPathThreads / 32);
    long long found = 0;
    for (long long gi = (long long)blockIdx.x * (kPathThreads / 32) + (threadIdx.x >> 5);
         gi < groups; gi += nwarps) {
        const long long w = gi * 32 + lane;
        uint32_t word = 0u;
        if (w < words) {
            word = __ldcg(P.mark + w);
            if (word) {
                P.mark[w] = 0u;
                P.vis[w] = __ldcg(P.vis + w) | word;
            }
        }
        found += __popc(word);
        while (__any_sync(0xffffffffu, word != 0u)) {
            const bool has = word != 0u;
            long long deg = 0, row = 0;
            int32_t v = 0;
            if (has) {
                v = (int32_t)(w * 32 + __ffs(word) - 1);
                word &= word - 1u;
                P.hops[v] = level + 1;
                const long long b = __ldg(P.off + v), e = __ldg(P.off + v + 1);
                if (b < 0 || e < b || e > P.nnz) P.ctl->bad = 1;
                else { deg = e - b; row = b; }
            }
            const unsigned long long x = deg > 0 ? (1ull << kPackShift) + (unsigned long long)deg : 0ull;
            const unsigned long long incl = warp_incl_scan(x);
            const unsigned long long tot = __shfl_sync(0xffffffffu, incl, 31);
            unsigned long long base = 0ull;
            if (lane == 31 && tot != 0ull) base = atomicAdd(&P.ctl->packed[nxt], tot);
            base = __shfl_sync(0xffffffffu, base, 31);
            if (deg > 0) {
                const unsigned long long ex = incl - x;
                const long long pos = (long long)(base >> kPackShift) + (long long)(ex >> kPackShift);
                if (pos < P.n) {
                    const long long eo = (long long)(base & kPackMask) + (long long)(ex & kPackMask);
                    P.qv[nxt][pos] = v;
                    P.qe[nxt][pos] = eo;
                    P.qk[nxt][pos] = row - eo;
                    mark_tiles(P, nxt, pos, eo, deg);
                } else {
                    P.ctl->bad = 1;
                }
            }
        }
    }
    found = warp_incl_scan(found);
    if (lane == 31 && found > 0) {
        atomicAdd(&P.ctl->reached, (unsigned long long)found);
        atomicMax(&P.ctl->levels, level + 2);
    }
}

__global__ void __launch_bounds__(kPathThreads, kPathMinBlocks)
paths_persistent(const __grid_constant__ PathParams P) {
    const long long nthreads = (long long)gridDim.x * kPathThreads;
    const long long tid = (long long)blockIdx.x * kPathThreads + threadIdx.x;
    for (long long i = tid; i < P.n; i += nthreads) {
        P.hops[i] = i == P.root ? 0 : -1;
        P.sigma[i] = i == P.root ? 1.0 : 0.0;
    }
    const long long words = (P.n + 31) / 32;
    for (long long i = tid; i < words; i += nthreads) {
        P.vis[i] = 0u;
        P.mark[i] = 0u;
    }
    __shared__ unsigned long long epoch;
    if (threadIdx.x == 0) epoch = 0ull;
    if (path_barrier(P, epoch)) {
        if (tid == 0) {
            const int32_t r = P.root;
            P.vis[r >> 5] = 1u << (r & 31);
            const long long b = P.off[r], e = P.off[r + 1];
            long long deg = 0;
            if (b < 0 || e < b || e > P.nnz) P.ctl->bad = 1;
            else deg = e - b;
            if (deg > 0) {
                P.qv[0][0] = r;
                P.qe[0][0] = 0;
                P.qk[0][0] = b;
                mark_tiles(P, 0, 0, 0, deg);
                P.ctl->packed[0] = (1ull << kPackShift) + (unsigned long long)deg;
            }
            P.ctl->reached = 1;
            P.ctl->levels = 1;
        }
        bool ok = path_barrier(P, epoch);
        for (int level = 0; ok; ++level) {
            const int cur = level & 1, nxt = cur ^ 1;
            const unsigned long long pk = __ldcg(&P.ctl->packed[cur]);
            const long long cnt = min((long long)(pk >> kPackShift), P.n);
            const long long E = (long long)(pk & kPackMask);
            if (cnt == 0) break;
            if (tid == 0) {
                P.ctl->edges += (unsigned long long)E;
                P.ctl->packed[nxt] = 0ull;   // last read at the start of level - 1
            }
            expand_paths(P, cur, cnt, E);
            if (!path_barrier(P, epoch)) break;
            collect_paths(P, level, nxt);
            ok = path_barrier(P, epoch);
        }
    }
    // last CTA out resets the barrier state for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&P.ctl->exit_count, 1u) + 1u == gridDim.x) {
            P.ctl->exit_count = 0u;
            P.ctl->arrived = 0ull;
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
    if (nnz >= (1ll << kPackShift)) {
        set_error("paths: nnz must be below 2^34");
        return BFS_ERR_UNSUPPORTED;
    }
    if (root < 0 || root >= n) {
        set_error("paths: root out of range");
        return BFS_ERR_ROOT_RANGE;
    }
    TraceRange tr("bfs_run_paths", root);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const int dv = ctx->device;
    if (!on_device(row_off, dv) || (nnz > 0 && !on_device(col, dv)) ||
        (weight && !on_device(weight, dv)) || !on_device(hops, dv) || !on_device(sigma, dv)) {
        set_error("paths: every array must be device memory of the context's GPU");
        return BFS_ERR_INVALID_ARG;
    }
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, paths_persistent, kPathThreads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "paths: occupancy query");
    if (nb < 1) {
        set_error("paths: traversal kernel cannot be resident");
        return BFS_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceAllocator* m = ctx->mem;
    const size_t nz = (size_t)n;
    const size_t words = (nz + 31) / 32 + 8;
    PathParams P;
    std::memset(&P, 0, sizeof(P));
    const size_t tiles = (size_t)nnz / kPathTile + 2;
    void* blk[11] = {m->alloc(nz * 4 + 64), m->alloc(nz * 4 + 64), m->alloc(nz * 8 + 64),
                     m->alloc(nz * 8 + 64), m->alloc(words * 4), m->alloc(words * 4),
                     m->alloc(sizeof(PathCtl)), m->alloc(tiles * 4), m->alloc(tiles * 4),
                     m->alloc(nz * 8 + 64), m->alloc(nz * 8 + 64)};
    auto release = [&]() {
        for (void* b : blk) m->release(b);
    };
    for (void* b : blk)
        if (!b) {
            release();
            set_error("paths: device memory exhausted");
            return BFS_ERR_NO_MEMORY;
        }
    P.qv[0] = static_cast<int32_t*>(blk[0]);
    P.qv[1] = static_cast<int32_t*>(blk[1]);
    P.qe[0] = static_cast<int64_t*>(blk[2]);
    P.qe[1] = static_cast<int64_t*>(blk[3]);
    P.vis = static_cast<uint32_t*>(blk[4]);
    P.mark = static_cast<uint32_t*>(blk[5]);
    P.ctl = static_cast<PathCtl*>(blk[6]);
    P.qc[0] = static_cast<int32_t*>(blk[7]);
    P.qc[1] = static_cast<int32_t*>(blk[8]);
    P.qk[0] = static_cast<int64_t*>(blk[9]);
    P.qk[1] = static_cast<int64_t*>(blk[10]);
    P.qc_cap = (long long)tiles;
    P.off = row_off;
    P.col = col;
    P.weight = weight;
    P.lo = w_lo;
    P.hi = w_hi;
    P.n = n;
    P.nnz = nnz;
    P.root = root;
    P.hops = hops;
    P.sigma = sigma;
    P.timeout_ns = 2000000000ll;
    e = cudaMemsetAsync(P.ctl, 0, sizeof(PathCtl), s);
    if (e == cudaSuccess) {
        void* args[] = {&P};
        e = cudaLaunchCooperativeKernel((const void*)paths_persistent, dim3(nb * ctx->sms),
                                        dim3(kPathThreads), args, 0, s);
    }
    PathCtl h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, P.ctl, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "paths traversal");
    if (h.bad) {
        set_error("paths: a row offset or column index lies outside the CSR");
        return BFS_ERR_INVALID_GRAPH;
    }
    if (h.status) {
        set_error("paths: a device-side grid barrier wait timed out");
        return BFS_ERR_TIMEOUT;
    }
    if (stats) {
        stats->levels = h.levels;
        stats->reached = (int64_t)h.reached;
        stats->edges_scanned = (int64_t)h.edges;
    }
    return BFS_OK;
}
