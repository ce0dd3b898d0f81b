// bfs_static.cu -- bfs_run_static: the single-source traversal for callers
// that must not allocate device memory.
//
// Everything the traversal needs besides the caller's CSR and outputs (the
// visited bitmap, the two frontier queues of every degree bin with their
// chunk tables, the level/barrier/status control block and the CSR check's
// result word) lives in one file-scope __device__ array of fixed size,
// reserved when the library's device code is loaded on a GPU and held until
// the process exits.  Host code never touches that array by name: its device
// address is looked up per device with cudaGetSymbolAddress and passed to the
// kernels.
//
// Each call first checks the CSR on the device (offsets non-decreasing
// inside [0, nnz], every column index inside [0, n)); the traversal kernel
// reads the check's result before its first access to the graph and ends
// at once when the check failed, so a bad index is never dereferenced.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bfs_runtime.h"

namespace bfs {

namespace lean {
const void* plain_persistent_fn(int mb);
}

namespace {

constexpr int64_t kStaticMaxVertices = 1ll << 19;   // 524,288 vertices
constexpr int64_t kStaticMaxEntries = 1ll << 25;    // 33,554,432 adjacency entries
constexpr int32_t kStaticTSmall = 32, kStaticTLarge = 2048;
constexpr int32_t kStaticChunkWarp = 1024, kStaticChunkCta = 8192;

constexpr size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kCtlBytes = a256(3 * sizeof(LevelCtl));
constexpr size_t kBarBytes = a256(sizeof(GridBarrier));
constexpr size_t kStatBytes = a256(sizeof(DevStats));
constexpr size_t kCheckBytes = a256(sizeof(int));   // the CSR check's result
constexpr size_t kControlBytes = kCtlBytes + kBarBytes + kStatBytes + kCheckBytes;
constexpr size_t kVisitedBytes = a256((size_t)(kStaticMaxVertices / 32 + 8) * 4);
constexpr size_t kQueueEntries = (size_t)kStaticMaxVertices + 1;
constexpr size_t kChunkCap1 = (size_t)(kStaticMaxEntries / kStaticChunkWarp) + 2;
constexpr size_t kChunkCap2 = (size_t)(kStaticMaxEntries / kStaticChunkCta) + 2;
constexpr size_t kParityBytes = a256(kQueueEntries * 4) +                                   // bin 0
                                a256(kQueueEntries * 4) + a256(kQueueEntries * 8) + a256(kChunkCap1 * 4) +  // bin 1
                                a256(kQueueEntries * 4) + a256(kQueueEntries * 8) + a256(kChunkCap2 * 4);   // bin 2
constexpr size_t kStaticScratchBytes = kControlBytes + kVisitedBytes + 2 * kParityBytes;

}  // namespace
}  // namespace bfs

// About 30 MB per GPU: the whole scratch of one traversal at the limits above.
static __device__ __align__(256) unsigned char g_bfs_static_scratch[bfs::kStaticScratchBytes];

namespace bfs {
namespace {

// Per-device set-up: the array's device address and the kernel's grid.  Only
// a successful set-up is cached, so a first call that failed (for instance
// one made during stream capture) is retried by the next call.
struct StaticDevice {
    std::mutex mu;
    bool ready = false;
    unsigned char* scratch = nullptr;   // device address of g_bfs_static_scratch
    int grid = 0;
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];

cudaError_t setup_device(StaticDevice& d, int dev) {
    std::lock_guard<std::mutex> lk(d.mu);
    if (d.ready) return cudaSuccess;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_bfs_static_scratch);
    int sms = 0, nb = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lean::plain_persistent_fn(2), kBlock, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    d.scratch = static_cast<unsigned char*>(p);
    d.grid = nb * sms;
    d.ready = true;
    return cudaSuccess;
}

// The CSR check: every offset pair in order, the first offset >= 0, the last
// <= nnz, every column index in [0, n).  Column indices are read 16 bytes at
// a time (col is 16-byte aligned), the tail one by one.
__global__ void static_csr_check(const int64_t* off, const int32_t* col, long long n,
                                 long long nnz, int* status) {
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (tid == 0) bad = off[0] < 0 || off[n] > nnz;
    for (long long v = tid; v < n; v += nthreads) bad |= off[v + 1] < off[v];
    const long long n4 = nnz / 4;
    const int4* c4 = reinterpret_cast<const int4*>(col);
    for (long long i = tid; i < n4; i += nthreads) {
        const int4 c = c4[i];
        bad |= (c.x < 0) | (c.x >= n) | (c.y < 0) | (c.y >= n) | (c.z < 0) | (c.z >= n) |
               (c.w < 0) | (c.w >= n);
    }
    for (long long e = 4 * n4 + tid; e < nnz; e += nthreads) bad |= col[e] < 0 || col[e] >= n;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(status, (int)kDevInvalidGraph);
}

}  // namespace
}  // namespace bfs

using namespace bfs;

extern "C" bfs_status bfs_run_static(const int64_t* row_off, const int32_t* col, int64_t n,
                                     int64_t nnz, int32_t root, int32_t* dist, int32_t* parent,
                                     void* stream, bfs_run_stats* stats) {
    if (!row_off || !dist || (!col && nnz > 0)) {
        set_error("bfs_run_static: null row_off, col or dist");
        return BFS_ERR_INVALID_ARG;
    }
    if (n < 1 || nnz < 0) {
        set_error("bfs_run_static: n must be >= 1 and nnz >= 0");
        return BFS_ERR_INVALID_ARG;
    }
    if (n > kStaticMaxVertices || nnz > kStaticMaxEntries) {
        set_error("bfs_run_static: graph exceeds the fixed scratch (at most 524288 vertices and "
                  "33554432 adjacency entries); use bfs_graph_upload + bfs_run instead");
        return BFS_ERR_UNSUPPORTED;
    }
    if (root < 0 || root >= n) {
        set_error("bfs_run_static: root out of range");
        return BFS_ERR_ROOT_RANGE;
    }
    if (col && (reinterpret_cast<uintptr_t>(col) & 15u)) {
        set_error("bfs_run_static: col must be 16-byte aligned");
        return BFS_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(row_off) & 7u) {
        set_error("bfs_run_static: row_off must be 8-byte aligned");
        return BFS_ERR_INVALID_ARG;
    }
    TraceRange tr("bfs_run_static", root);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("bfs_run_static: device index too large");
        return BFS_ERR_UNSUPPORTED;
    }
    StaticDevice& d = g_static_dev[dev];
    e = setup_device(d, dev);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: per-device set-up");
    if (d.grid < 1) {
        set_error("bfs_run_static: traversal kernel cannot be resident");
        return BFS_ERR_CUDA;
    }

    // carve the scratch: control | visited | parity 0 queues | parity 1 queues
    unsigned char* p = d.scratch;
    TraversalParams P;
    std::memset(&P, 0, sizeof(P));
    P.ctl = reinterpret_cast<LevelCtl*>(p);
    P.bar = reinterpret_cast<GridBarrier*>(p + kCtlBytes);
    P.stats = reinterpret_cast<DevStats*>(p + kCtlBytes + kBarBytes);
    int* check = reinterpret_cast<int*>(p + kCtlBytes + kBarBytes + kStatBytes);
    P.pre_status = check;
    p += kControlBytes;
    P.visited = reinterpret_cast<uint32_t*>(p);
    p += kVisitedBytes;
    for (int par = 0; par < 2; ++par) {
        for (int b = 0; b < kBins; ++b) {
            BinQueue& Q = P.q[par][b];
            Q.cap = n + 1;
            Q.v = reinterpret_cast<int32_t*>(p);
            p += a256(kQueueEntries * 4);
            if (b > 0) {
                const int64_t C = b == 1 ? kStaticChunkWarp : kStaticChunkCta;
                Q.eoff = reinterpret_cast<int64_t*>(p);
                p += a256(kQueueEntries * 8);
                Q.chunk = reinterpret_cast<int32_t*>(p);
                Q.chunk_cap = (nnz + C - 1) / C + 2;
                p += a256((b == 1 ? kChunkCap1 : kChunkCap2) * 4);
            }
        }
    }
    P.n = n;
    P.nnz = nnz;
    P.bu_limit = n;
    P.off = row_off;
    P.col = col;
    P.t_small = kStaticTSmall;
    P.t_large = kStaticTLarge;
    P.chunk_warp = kStaticChunkWarp;
    P.chunk_cta = kStaticChunkCta;
    P.dist = dist;
    P.parent = parent;
    P.root_caller = root;
    P.timeout_ns = 2000000000ll;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the control block (with the check's result word) must start at zero;
    // the traversal kernel clears the bitmap
    e = cudaMemsetAsync(d.scratch, 0, kControlBytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: clearing the control block");
    static_csr_check<<<d.grid, kBlock, 0, s>>>(row_off, nnz > 0 ? col : nullptr, n, nnz, check);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: CSR check launch");
    void* args[] = {&P};
    e = cudaLaunchCooperativeKernel(lean::plain_persistent_fn(2), dim3(d.grid), dim3(kBlock), args, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: cooperative launch");
    if (!stats) return BFS_OK;
    DevStats h;
    e = cudaMemcpyAsync(&h, P.stats, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: traversal");
    stats->levels = h.levels;
    stats->reached = h.reached;
    stats->edges_scanned = h.edges;
    stats->status = h.status;
    stats->bottom_up_levels = h.bu_levels;
    if (h.status == kDevTimeout) {
        set_error("bfs_run_static: device-side grid barrier wait timed out");
        return BFS_ERR_TIMEOUT;
    }
    if (h.status == kDevInvalidGraph) {
        set_error("bfs_run_static: CSR check failed (an offset decreases or lies outside "
                  "[0, nnz], or a column index lies outside [0, n))");
        return BFS_ERR_INVALID_GRAPH;
    }
    if (h.status != kDevOk) {
        set_error("bfs_run_static: device queue overflow (internal error)");
        return BFS_ERR_CUDA;
    }
    return BFS_OK;
}
